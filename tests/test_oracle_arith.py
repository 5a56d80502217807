"""Pins of the oracle's integer layer against definitions it does not use itself.

Each test checks the oracle against an independent statement of the same fact:
schoolbook products in Python integers, exact CRT, sympy's primality test, the
published SplitMix64 vector, brute-force root search.
"""
import json
import os
import random

import numpy as np
import pytest
import sympy

from oracle import _clib as C
from oracle import params as PP

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def small_params(logn=5, n_q=3):
    return PP.Params(logn, n_q, 2, 60, 40, 60)


def py_negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return [x % q for x in out]


@pytest.mark.parametrize("logn", [1, 2, 3, 5, 6])
def test_ntt_is_evaluation_at_odd_roots(logn):
    """forward NTT output i = a(psi^(2 rev(i) + 1)), evaluated here with Python ints"""
    P = PP.Params(max(logn, 1), 2, 1, 50, 40, 50)
    n = 1 << logn
    for q, psi in zip(P.q, P.psi_q):
        a = [random.randrange(q) for _ in range(n)]
        got = C.ntt_forward(np.array([a], dtype=np.uint64), [q], [psi], logn)[0]
        for i in range(n):
            rev = int(format(i, "0%db" % logn)[::-1], 2) if logn else 0
            root = pow(psi, 2 * rev + 1, q)
            want = sum(a[j] * pow(root, j, q) for j in range(n)) % q
            assert int(got[i]) == want
        back = C.ntt_inverse(np.array([got], dtype=np.uint64), [q], [psi], logn)[0]
        assert [int(x) for x in back] == a
        # the oracle's own O(N^2) routine agrees too
        assert (C.ntt_naive(np.array(a, dtype=np.uint64), q, psi, logn) == got).all()


@pytest.mark.parametrize("logn", [3, 6, 8])
def test_ntt_product_is_negacyclic_convolution(logn):
    P = PP.Params(logn, 2, 1, 60, 40, 60)
    n = 1 << logn
    q, psi = P.q[0], P.psi_q[0]
    a = [random.randrange(q) for _ in range(n)]
    b = [random.randrange(q) for _ in range(n)]
    A = C.ntt_forward(np.array([a], dtype=np.uint64), [q], [psi], logn)
    B = C.ntt_forward(np.array([b], dtype=np.uint64), [q], [psi], logn)
    prod = C.ntt_inverse(C.mul(A, B, [q]), [q], [psi], logn)[0]
    assert [int(x) for x in prod] == py_negacyclic(a, b, q)
    if logn <= 6:
        nv = C.negacyclic_naive(np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64), q)
        assert [int(x) for x in nv] == py_negacyclic(a, b, q)


def test_primes_and_roots():
    for P in (PP.cfg1_params(), PP.Params(10, 24, 3, 60, 42, 60, h=64, n_p=7, boot_bits=48, n_boot=14)):
        allp = list(P.q) + list(P.p)
        assert len(set(allp)) == len(allp)
        for q, psi in zip(allp, P.psi_q + P.psi_p):
            assert sympy.isprime(q)
            assert q % (2 * P.n) == 1
            assert pow(psi, P.n, q) == q - 1
        assert P.q[0].bit_length() == P.q0_bits
        assert all(p.bit_length() == P.p_bits for p in P.p)
        # q0 is the largest NTT-friendly prime below 2^q0_bits
        for k in range(P.q[0] // (2 * P.n) + 1, ((1 << P.q0_bits) - 1) // (2 * P.n) + 1):
            assert not sympy.isprime(k * 2 * P.n + 1)


def test_smallest_root_brute_force():
    for q, n in ((97, 8), (193, 16), (7681, 256), (12289, 512)):
        brute = min(x for x in range(2, q) if pow(x, n, q) == q - 1)
        assert PP.smallest_primitive_root_2n(q, n) == brute


def test_scale_ladder():
    """Delta_{l-1} = Delta_l^2 / q_l inside each segment, each Delta within 2^-8 of 2^bits"""
    P = PP.Params(10, 24, 3, 60, 42, 60, h=64, n_p=7, boot_bits=48, n_boot=14)
    c = P.n_circuit
    for l in range(1, P.L + 1):
        if l == c + 1:
            assert P.delta[c] == 2.0 ** 42
            continue
        assert P.delta[l - 1] == (P.delta[l] * P.delta[l]) / float(P.q[l])
    for l in range(P.n_q):
        bits = 42 if l <= c else 48
        assert abs(np.log2(P.delta[l]) - bits) < 2 ** -8


def test_base_convert_is_crt_plus_small_multiple():
    P = small_params(4, 3)
    qin = list(P.q)
    qout = list(P.p)
    n = P.n
    Q = qin[0] * qin[1] * qin[2]
    x = [random.randrange(Q) for _ in range(n)]
    xin = np.array([[v % qi for v in x] for qi in qin], dtype=np.uint64)
    y = C.base_convert(xin, qin, qout)
    for j in range(n):
        ok = False
        for u in range(len(qin)):
            if all(int(y[m, j]) == (x[j] + u * Q) % qout[m] for m in range(len(qout))):
                ok = True
        assert ok


def test_rescale_is_rounded_division():
    P = small_params(4, 4)
    q = list(P.q)
    Q = q[0] * q[1] * q[2] * q[3]
    n = P.n
    x = [random.randrange(Q) for _ in range(n)]
    xin = np.array([[v % qi for v in x] for qi in q], dtype=np.uint64)
    out = C.rescale(xin, q)
    for j in range(n):
        v = x[j] if x[j] <= Q // 2 else x[j] - Q       # centred
        r = v % q[3]
        if r > q[3] // 2:
            r -= q[3]
        want = (v - r) // q[3]                           # = round(v / q_l)
        assert abs(want * q[3] - v) <= q[3] // 2
        for i in range(3):
            assert int(out[i, j]) == want % q[i]


def test_mod_down_divides_by_P():
    P = PP.Params(4, 2, 1, 60, 40, 60, n_p=2)
    q, p = list(P.q), list(P.p)
    Q, Pm = q[0] * q[1], p[0] * p[1]
    n = P.n
    x = [random.randrange(Q * Pm) for _ in range(n)]
    xin = np.array([[v % m for v in x] for m in q + p], dtype=np.uint64)
    out = C.mod_down(xin, q, p)
    for j in range(n):
        # exact CRT of the output, centred mod Q, times P, is within (np + 1) * P of x
        v = (int(out[0, j]) * q[1] * pow(q[1], -1, q[0]) + int(out[1, j]) * q[0] * pow(q[0], -1, q[1])) % Q
        diff = (v * Pm - x[j]) % (Q * Pm)
        diff = diff - Q * Pm if diff > Q * Pm // 2 else diff
        assert abs(diff) <= (len(p) + 1) * Pm


def test_mod_raise_and_automorphism():
    P = small_params(4, 3)
    q = list(P.q)
    n = P.n
    c = np.array([random.randrange(q[0]) for _ in range(n)], dtype=np.uint64)
    up = C.mod_raise(c, q)
    for j in range(n):
        v = int(c[j]) if int(c[j]) <= q[0] // 2 else int(c[j]) - q[0]
        assert all(int(up[i, j]) == v % q[i] for i in range(3))
    # a(X^g) by direct substitution
    a = [random.randrange(q[1]) for _ in range(n)]
    for g in (5, 25, 2 * n - 1):
        want = [0] * n
        for i, ai in enumerate(a):
            k = i * g % (2 * n)
            if k < n:
                want[k] = (want[k] + ai) % q[1]
            else:
                want[k - n] = (want[k - n] - ai) % q[1]
        got = C.automorphism(np.array([a], dtype=np.uint64), [q[1]], g, P.logn)[0]
        assert [int(x) for x in got] == want


def test_splitmix_published_vector():
    gold = json.load(open(os.path.join(GOLD, "splitmix64_seed0.json")))
    want = [int(h, 16) for h in gold["outputs_hex"]]
    # stream_word(key, i) is the i-th output of SplitMix64 started from state `key`
    assert [C.stream_word(0, i) for i in range(3)] == want


def test_samplers():
    n = 1 << 14
    t = C.sample_ternary(n, 9, 77)
    assert set(np.unique(t)) <= {-1, 0, 1}
    assert abs((t == 0).mean() - 1 / 3) < 0.03
    h = C.sample_hw(n, 192, 9, 1, 2)
    assert (h != 0).sum() == 192 and set(np.unique(h)) <= {-1, 0, 1}
    g = C.sample_gauss(n, 3.2, 9, 5)
    assert np.abs(g).max() <= 19
    assert abs(g.std() - 3.2) < 0.1 and abs(g.mean()) < 0.1
    tab = C.gauss_table(3.2)
    assert (np.diff(tab.astype(np.float64)) >= 0).all() and int(tab[-1]) == 1 << 63
    # symmetric table: P(e <= -k-1) == P(e >= k+1)
    for k in range(19):
        lo = int(tab[18 - k])
        hi = (1 << 63) - int(tab[19 + k])
        assert abs(lo - hi) <= 1 << 12   # one double ulp at 2^63
    q = [(1 << 61) - 1, 1152921504606830593]
    u = C.sample_uniform(q, [0, 5], n, 3, 4)
    assert (u[0] < q[0]).all() and (u[1] < q[1]).all()
    assert abs(u[1].astype(np.float64).mean() / q[1] - 0.5) < 0.02
    # the same limb id gives the same values whatever the limb's position
    u2 = C.sample_uniform([q[1]], [5], n, 3, 4)
    assert (u2[0] == u[1]).all()
