"""The algorithmic work counts behind the bench's roofline figures, checked by enumeration (CPU).

M2L per unordered cell pair: the auxiliary recurrence (3 C(p+4,4) flops) and, per direction and
local-expansion class, the contraction terms with |n| + |j| <= p, less those of L^0 when only
accelerations are requested, 2 flops each.  P2P: 25 flops per unordered particle pair for both
accelerations.
"""
import itertools
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
import bench  # noqa: E402


def _mis(order):
    return [m for m in itertools.product(range(order + 1), repeat=3) if sum(m) <= order]


def test_contraction_term_counts():
    from math import comb
    for p in range(1, 9):
        mis = _mis(p)
        terms = sum(1 for n in mis for j in mis if sum(n) + sum(j) <= p)
        assert terms == comb(p + 6, 6)
        assert sum(1 for n in mis for j in mis if sum(n) + sum(j) <= p and sum(n) == 0) == comb(p + 3, 3)


def test_m2l_flops_at_the_benchmark_order():
    # p = 6: 3 C(10,4) = 630 for D, 2 directions x 2 flops x (924 - 84) = 3360 per class
    assert bench.m2l_flops(6, 1, {}) == 630 + 3360
    assert bench.m2l_flops(6, 10, {"m2l_class_pairs": 20}) == 10 * 630 + 20 * 3360


def test_p2p_flops_per_pair():
    # 3 differences, r^2 (1 mul + 2 FMA = 5), rsqrt, r^-3 (2 mul), 2 mass products, 6 FMA (12)
    assert bench.P2P_FLOPS_PER_PAIR == 3 + 5 + 1 + 2 + 2 + 12


def test_traffic_record_kept_only_while_its_source_matches(tmp_path, monkeypatch):
    # the DRAM bytes of a capture are reported only while the kernel source hashes as it did then
    import hashlib
    import json
    src = tmp_path / "kern.cuh"
    src.write_text("kernel v1\n")
    (tmp_path / "profiles").mkdir()
    rec = {"bytes_per_launch": 4.0e9, "units_per_launch": 2.0e10, "unit": "pairs", "source": str(src),
           "source_sha256_16": hashlib.sha256(b"kernel v1\n").hexdigest()[:16]}
    (tmp_path / "profiles" / "roofline_traffic.json").write_text(json.dumps({"note": "x", "p2p": rec}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.captured_traffic()
    assert set(got) == {"p2p"}
    # scaled by the units of the bench's own launch
    assert bench.scaled_traffic(got, "p2p", 1.0e10) == 2.0e9
    assert bench.scaled_traffic(got, "m2l", 1.0e10) is None
    src.write_text("kernel v2\n")
    assert bench.captured_traffic() == {}


def test_committed_traffic_records_name_existing_sources():
    import json
    data = json.load(open(os.path.join(os.path.dirname(HERE), "profiles", "roofline_traffic.json")))
    for key, rec in data.items():
        if not isinstance(rec, dict):
            continue
        assert rec["bytes_per_launch"] > 0 and rec["units_per_launch"] > 0, key
        for part in rec["source"].split("+"):
            assert os.path.isfile(os.path.join(os.path.dirname(HERE), part)), part
