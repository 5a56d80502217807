"""The arithmetic behind base conversion on the tensor cores, checked on the CPU: cutting the
input words and the pre-shifted table entries into 8-bit chunks turns sum_i x_i c_i mod p into
eight FP32 matrix-product columns whose values are exact integers below 2^23; accumulating them
from a start value of 2^23 keeps every partial sum an exact integer in [2^23, 2^24), so the final
word's low 23 bits are the column sum, from which the sum is reassembled mod p as
lo + 2^24 hi (lo = D_0 + 2^8 D_1 + 2^16 D_2 < 2^39)."""
import numpy as np

rng = np.random.default_rng(23)


def _chunks(v):
    return [(v >> (8 * a)) & 0xFF for a in range(8)]


def _convert_by_chunks(x, c, p):
    """x: nin words, c: nin table entries (mod p); returns y = sum_i x_i c_i mod p through the
    chunked FP16 x FP16 -> FP32 product"""
    nin = len(x)
    A = np.array([ch for xi in x for ch in _chunks(xi)], dtype=np.float16)          # K = 8 nin
    B = np.zeros((8, 8 * nin), dtype=np.float16)
    for i, ci in enumerate(c):
        for a in range(8):
            e = (ci << (8 * a)) % p
            for b, ch in enumerate(_chunks(e)):
                B[b, 8 * i + a] = ch
    D = np.full(8, 2.0 ** 23, dtype=np.float32)   # FP32 accumulation from 2^23, one product at a time
    for k in range(8 * nin):
        D = (D + A[k].astype(np.float32) * B[:, k].astype(np.float32)).astype(np.float32)
    assert (D < 2.0 ** 24).all()
    w = [int(v) for v in D.view(np.uint32)]
    assert all(v >> 23 == 0x4B000000 >> 23 for v in w)
    d = [v - 0x4B000000 for v in w]
    lo = d[0] + (d[1] << 8) + (d[2] << 16)
    hi = d[3] + (d[4] << 8) + (d[5] << 16) + (d[6] << 24) + (d[7] << 32)
    assert lo < 2 ** 39 and hi < 2 ** 56
    return (lo + (hi << 24)) % p


def test_chunked_conversion_equals_the_sum():
    for nin, bits in ((8, 60), (7, 60), (16, 60), (3, 42), (1, 48)):
        p = int(rng.integers(2 ** (bits - 1), 2 ** bits)) | 1
        x = [int(v) for v in rng.integers(0, 2 ** 61, nin, dtype=np.uint64)]
        c = [int(v) % p for v in rng.integers(0, 2 ** 62, nin, dtype=np.uint64)]
        assert _convert_by_chunks(x, c, p) == sum(a * b for a, b in zip(x, c)) % p


def test_largest_chunk_sums_stay_exact():
    """every chunk 255 on both sides with 16 inputs (K = 128): each column sum is 128 * 255^2,
    still below 2^23"""
    assert 128 * 255 * 255 < 2 ** 23
    p = (1 << 61) - 1
    x = [2 ** 64 - 1] * 16
    A = np.full(128, 255, dtype=np.float32)
    assert float(np.sum(A * A, dtype=np.float32)) == 128 * 255 * 255
    c = [p - 1] * 16
    assert _convert_by_chunks(x, c, p) == sum(a * b for a, b in zip(x, c)) % p


def _round_term(xh, q):
    """one term of the exact conversion's rounding sum in 58-bit fixed point: 1/q = M 2^-(64+b),
    b = bitlen(q) - 1, M = floor(2^(64+b) / q); the 128-bit product xh M shifted right by b + 6"""
    b = q.bit_length() - 1
    m = (1 << (64 + b)) // q
    assert 2 ** 63 <= m < 2 ** 64
    return (xh * m) >> (b + 6)


def test_fixed_point_rounding_term_within_bound():
    """the fixed-point sum of up to 16 terms xh_i / q_i stays within 2^-53 of the exact sum and
    rounds to the same integer away from half-integers (the exact value is never a half-integer
    for odd moduli)"""
    from fractions import Fraction
    for trial in range(200):
        nin = int(rng.integers(1, 17))
        qs = [int(rng.integers(2 ** (int(rng.integers(40, 62)) - 1), 2 ** 61)) | 1 for _ in range(nin)]
        xs = [int(rng.integers(0, q)) for q in qs]
        if trial % 10 == 0:
            xs = [q - 1 for q in qs]                 # largest terms
        s = sum(_round_term(x, q) for x, q in zip(xs, qs))
        assert s < 2 ** 62
        exact = sum(Fraction(x, q) for x, q in zip(xs, qs))
        err = exact - Fraction(s, 2 ** 58)
        assert 0 <= err < Fraction(1, 2 ** 53)
        v = (s + 2 ** 57) >> 58
        if abs(exact - int(exact) - Fraction(1, 2)) > Fraction(1, 2 ** 52):
            assert v == int(exact + Fraction(1, 2))
