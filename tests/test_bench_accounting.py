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
