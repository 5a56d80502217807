"""Measurement arithmetic of bench.py, checked by hand on small cases (no GPU): the NTT's
butterfly count from its algorithmic bytes, the integer-multiply peak, and the DRAM ratios
taken from the ncu captures."""
import math

import bench


def test_ntt_butterflies_from_bytes():
    """one limb transform of N = 2^16: 16 stages of N/2 butterflies, 2 N 8 algorithmic bytes;
    the roofline divides the bytes by 2"""
    n = 1 << 16
    limbs = 10
    butterflies = limbs * 16 * n // 2
    bytes_ = limbs * 2 * n * 8
    stats = {"ntt_fwd": {"bytes": float(bytes_), "ms": 0.001, "launches": 2}}    # 1 us
    r = bench.ntt_alu_roofline(stats, {"sm_max_mhz": 2070.0})
    assert math.isclose(r["ntt_fwd"]["achieved"], butterflies / 1e-6 / 1e9, rel_tol=1e-3)


def test_integer_multiply_peak():
    """64 multiply lanes per SM per clock, 152 SMs, 16 lane-cycles per 64-bit Shoup
    butterfly (6 wide products counted twice + 4 narrow)"""
    assert bench.NTT_MUL_LANE_CYCLES_PER_BUTTERFLY == 6 * 2 + 4
    r = bench.ntt_alu_roofline({}, {"sm_max_mhz": 2000.0})
    assert math.isclose(r["peak"], 64 * 152 * 2000e6 / 16 / 1e9, rel_tol=1e-3)


def test_dram_ratios_from_captures():
    """NTT: two passes of 256 limbs read and wrote 491.3 MB for 268.4 MB of algorithmic bytes;
    key switch: 149.9 MB for 365 limbs of 512 KiB"""
    assert math.isclose(bench.NTT_FWD_DRAM_PER_ALGO_BYTE, 491.3 / 268.4, rel_tol=1e-3)
    assert math.isclose(bench.KS_DRAM_PER_ALGO_BYTE, 149.9 / (365 * 0.524288), rel_tol=1e-3)
    assert 1.0 < bench.NTT_FWD_DRAM_PER_ALGO_BYTE < 2.0 and 0.5 < bench.KS_DRAM_PER_ALGO_BYTE < 1.0
    # a 24-limb transform (in L2, warm): 0.163 MB of DRAM traffic for 25.2 MB of algorithmic bytes
    assert math.isclose(bench.NTT_FWD_DRAM_PER_ALGO_BYTE_IN_L2, 0.16256 / 25.165824, rel_tol=1e-6)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle on the host, no GPU needed) prints one JSON
    line with the keys the bench contract asks of that arm"""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "1", "--oracle-small"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["higher_is_better"] is False and line["unit"] == "ms"
    assert line["value"] > 0 and line["metric"] == bench.METRIC
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # every step of the block measured (three in the timed region, the rest outside it), and the
    # value is their sum
    st = line["stage_ms"]
    assert len(st) == line["config"]["steps_per_block"] >= 10
    assert abs(sum(st.values()) - line["value"]) <= 0.1 * len(st)
