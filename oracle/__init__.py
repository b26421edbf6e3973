"""Plain FP64 CPU oracle of the MGARD-style reduction path (Sec. IV-A, Alg. 1
and Sec. IV-B, Alg. 2 of the HPDR paper).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The oracle shares no code
with the GPU library and never imports it.

Functions whose result the paper and mathematics pin (see tests/test_oracle_*):
decompose / recompose (identity, multilinear invariance, dense L2-projection
brute force, closed forms), the adjoints (dot-product identity, dense
transposes), bins (error-bound property), Huffman (Kraft equality, optimal
total cost, brute-force optimality on small alphabets, round trip).
Parity unpinned (fixed only by the written definitions and the round-trip and
bound properties): the container layout, the tie-break of equal frequencies,
the choice of D and K.
"""
from .api import *  # noqa: F401,F403
