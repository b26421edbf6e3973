"""Host-side helpers of bench.py, CPU only: the roofline numerator
(algorithmic bytes per launch), level sizes, the source hashes that key the
ncu traffic table, and the table's lookup."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.argv = sys.argv[:1]

import bench  # noqa: E402


def test_level_sizes():
    assert bench.level_nodes((513, 513, 513), 0) == 513 ** 3
    assert bench.level_nodes((513, 513, 513), 1) == 257 ** 3
    # one coarsening keeps the even positions plus the last node
    assert bench.level_nodes((500,), 1) == 251 and bench.level_nodes((501,), 1) == 251
    assert bench.level_nodes((500, 100), 2) == 126 * 26


def test_algorithmic_bytes_of_the_finest_level():
    """513^3 FP32: read the level (4 B/node), write a symbol per new node
    (2 B), b and the coarse copy (4 B each per coarse node)."""
    NL, NL1 = 513 ** 3, 257 ** 3
    new = NL - NL1
    assert bench.algorithmic_bytes("c_restrict_quant_L", 4, NL, NL1, 0, 0) == 4 * NL + 2 * new + 8 * NL1 == 911881740
    assert bench.algorithmic_bytes("d_restrict_sym_L", 4, NL, NL1, 0, 0) == 2 * new + 4 * NL1
    assert bench.algorithmic_bytes("d_expand_L", 4, NL, NL1, 0, 0) == 2 * new + 4 * NL1 + 4 * NL
    assert bench.algorithmic_bytes("d_decode", 4, NL, NL1, 8e8, 1000) == 1e8 + 8000 + 2 * NL
    assert bench.algorithmic_bytes("no_such_group", 4, NL, NL1, 0, 0) is None


def test_source_hashes_and_traffic_lookup():
    hl, hh = bench.source_hash("c_restrict_quant_L"), bench.source_hash("d_decode")
    assert re.fullmatch(r"[0-9a-f]{16}", hl) and re.fullmatch(r"[0-9a-f]{16}", hh) and hl != hh
    assert bench.source_hash("d_expand_L") == hl and bench.source_hash("c_encode") == hh
    # a row counts only when its hash is the current one; then its bytes are returned
    rows = {}
    for ln in open(os.path.join(ROOT, "profiles", "traffic.md")):
        parts = [p.strip() for p in ln.strip().strip("|").split("|")]
        if len(parts) >= 4 and re.fullmatch(r"[0-9a-f]{16}", parts[1]):
            rows[parts[0]] = (parts[1], float(parts[3]))
    assert rows, "traffic table has no rows"
    for group, (h, val) in rows.items():
        got = bench.ncu_traffic(group)
        if h == bench.source_hash(group):
            assert got == val
        else:
            assert got is None


def test_workload_name_names_shape_and_bound():
    name = bench.workload_name((513, 513, 513), 1e-3)
    assert name.startswith("513x513x513 FP32") and "rel Linf 0.001" in name
    assert bench.workload_name((500, 500, 100), 1e-2).startswith("500x500x100")
