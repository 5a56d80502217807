"""Mistakes planted in the oracle, on the CPU: each is a plausible slip in one step, and the
pin of that step must fail on it (while the same pin passes on a correct restatement), so
the pins would notice such a slip in the oracle itself."""
import math

import numpy as np
import pytest

from oracle import _clib as C
from oracle import params as PP
from oracle.scheme import Oracle
from tests import test_oracle_arith as A
from tests import test_oracle_scheme as S


def _rescale_py(c, q, centred):
    """(c_i - r) q_l^{-1} mod q_i, r the remainder of the top limb, centred or in [0, q_l)"""
    c = np.asarray(c, dtype=np.uint64)
    l = c.shape[0] - 1
    ql = int(q[l])
    out = np.empty((l, c.shape[1]), dtype=np.uint64)
    for i in range(l):
        qi = int(q[i])
        inv = pow(ql, -1, qi)
        row = []
        for a, t in zip(c[i], c[l]):
            r = int(t) - ql if centred and int(t) > ql // 2 else int(t)
            row.append(((int(a) - r) * inv) % qi)
        out[i] = row
    return out


def _base_convert_py(x, qin, qout, terms):
    """sum over the first `terms` inputs of [x_i qhat_i^{-1}]_{q_i} qhat_i, mod each output"""
    x = np.asarray(x, dtype=np.uint64)
    Q = math.prod(int(v) for v in qin)
    out = np.zeros((len(qout), x.shape[1]), dtype=np.uint64)
    for m, p in enumerate(qout):
        for j in range(x.shape[1]):
            s = 0
            for i in range(terms):
                qh = Q // int(qin[i])
                s += (int(x[i, j]) * pow(qh, -1, int(qin[i])) % int(qin[i])) * qh
            out[m, j] = s % int(p)
    return out


def test_uncentred_rescale_fails_its_pin(monkeypatch):
    monkeypatch.setattr(C, "rescale", lambda c, q: _rescale_py(c, q, centred=True))
    A.test_rescale_is_rounded_division()                         # correct restatement passes
    monkeypatch.setattr(C, "rescale", lambda c, q: _rescale_py(c, q, centred=False))
    with pytest.raises(AssertionError):
        A.test_rescale_is_rounded_division()


def test_base_conversion_with_a_dropped_term_fails_its_pin(monkeypatch):
    monkeypatch.setattr(C, "base_convert", lambda x, qi, qo: _base_convert_py(x, qi, qo, len(qi)))
    A.test_base_convert_is_crt_plus_small_multiple()             # correct restatement passes
    monkeypatch.setattr(C, "base_convert", lambda x, qi, qo: _base_convert_py(x, qi, qo, len(qi) - 1))
    with pytest.raises(AssertionError):
        A.test_base_convert_is_crt_plus_small_multiple()


def test_rotation_in_the_wrong_direction_fails_its_pin(monkeypatch):
    """Galois element 5^{-r} instead of 5^r (keys generated for the same wrong elements, so
    everything decrypts): the slot-roll pin sees the wrong direction"""
    monkeypatch.setattr(Oracle, "galois", lambda self, r: pow(5, (-r) % (self.P.n // 2), 2 * self.P.n))
    o = Oracle(PP.Params(9, 6, 3, 60, 40, 60, h=32), 42)
    o.gen_relin_key()
    o.gen_conj_key()
    o.gen_rotation_keys([1, 3, 7, 100])
    with pytest.raises(AssertionError):
        S.test_rotation_conjugation_product(o)


def test_ntt_with_the_inverse_root_or_natural_order_fails_its_pin(monkeypatch):
    """psi^{-1} for psi evaluates at the same set of odd powers, only permuted; an output in
    natural instead of bit-reversed order is the same values permuted too: the pin checks
    each output position"""
    real = C.ntt_forward
    logn = 5
    rev = np.array([int(format(i, "05b")[::-1], 2) for i in range(1 << logn)])
    monkeypatch.setattr(C, "ntt_forward", lambda a, q, psi, lg: real(
        a, q, [pow(int(p), -1, int(m)) for p, m in zip(psi, q)], lg))
    with pytest.raises(AssertionError):
        A.test_ntt_is_evaluation_at_odd_roots(logn)
    monkeypatch.setattr(C, "ntt_forward", lambda a, q, psi, lg: real(a, q, psi, lg)[:, rev])
    with pytest.raises(AssertionError):
        A.test_ntt_is_evaluation_at_odd_roots(logn)
    monkeypatch.setattr(C, "ntt_forward", real)
    A.test_ntt_is_evaluation_at_odd_roots(logn)


def _kernel_vector_py(K, w, flip_offsets=False, wrap_sign=-1.0):
    """Fig. 1 kernel vector; flip_offsets turns the cross-correlation into a convolution,
    wrap_sign = +1 forgets the sign of a tap that wraps around Y^{w^2} + 1"""
    f = K.shape[0]
    c = f // 2
    n = w * w
    v = np.zeros(n)
    for a in range(f):
        for b in range(f):
            q = -((a - c) * w + (b - c))
            if flip_offsets:
                q = -q
            if q >= 0:
                v[q] += K[a, b]
            else:
                v[n + q] += wrap_sign * K[a, b]
    return v


def test_conv_kernel_vector_slips_fail_their_pin(monkeypatch):
    from oracle import encoding as E
    from tests import test_oracle_encoding as EN
    monkeypatch.setattr(E, "kernel_vector", lambda K, w: _kernel_vector_py(K, w))
    EN.test_conv2d_as_negacyclic_convolution()                   # correct restatement passes
    for slip in (dict(flip_offsets=True), dict(wrap_sign=1.0)):
        monkeypatch.setattr(E, "kernel_vector", lambda K, w, s=slip: _kernel_vector_py(K, w, **s))
        with pytest.raises(AssertionError):
            EN.test_conv2d_as_negacyclic_convolution()


def test_dft_twiddle_root_slip_fails_its_pin(monkeypatch):
    """W_k of the block B_k with omega_{4k} (Eq. 2's subscript copied to the block size) in
    place of omega_{8k}: the recursive factorisation no longer rebuilds T = V P"""
    from oracle import encoding as E
    from tests import test_oracle_encoding as EN
    monkeypatch.setattr(E, "W_diag", lambda k: np.array([E.omega(4 * k, pow(5, i, 4 * k)) for i in range(k)]))
    with pytest.raises(AssertionError):
        EN.test_special_dft_factorisation(16)


def _div_round_py(self, acc, level, S, mode="centred"):
    """(a - r) M^{-1} mod q_i over the first `level` Q rows, M = prod S, r the remainder of a
    mod M by exact CRT: centred (the rounding), in [0, M) (a floor), or centred plus one unit"""
    M = math.prod(int(m) for m in S)
    out = np.empty((level, acc.shape[1]), dtype=np.uint64)
    for j in range(acc.shape[1]):
        r = 0
        for k, mk in enumerate(S):
            mk = int(mk)
            r += int(acc[level + k, j]) * pow((M // mk) % mk, -1, mk) * (M // mk)
        r %= M
        if mode != "floor" and r > M // 2:
            r -= M
        for i in range(level):
            qi = int(self.P.q[i])
            v = (int(acc[i, j]) - r) * pow(M % qi, -1, qi)
            if mode == "plus_one":
                v += 1
            out[i, j] = v % qi
    return out


def test_fused_rescale_slips_fail_their_pin(monkeypatch):
    """ModDown fused with the rescale taking the floor (remainder in [0, q_l P)) instead of the
    rounding, or landing one unit off: the rounded-division pin fails on both"""
    from tests import test_oracle_plain as PLT
    monkeypatch.setattr(Oracle, "_div_round", lambda self, a, l, S: _div_round_py(self, a, l, S))
    PLT.test_mod_down_rescale_is_rounded_division(2)             # correct restatement passes
    for mode in ("floor", "plus_one"):
        monkeypatch.setattr(Oracle, "_div_round", lambda self, a, l, S, m=mode: _div_round_py(self, a, l, S, m))
        with pytest.raises(AssertionError):
            PLT.test_mod_down_rescale_is_rounded_division(2)


def test_chebyshev_leaf_with_a_dropped_term_fails_its_pin(monkeypatch):
    """a Chebyshev leaf that forgets its highest term: the series pin against the plain
    term-by-term evaluation fails"""
    from tests import test_oracle_plain as PLT
    real = Oracle.cheb_leaf

    def dropped(self, T, at, coeffs):
        c = list(coeffs)
        for k in range(len(c) - 1, 0, -1):
            if c[k] != 0.0:
                c[k] = 0.0
                break
        return real(self, T, at, c)
    monkeypatch.setattr(Oracle, "cheb_leaf", dropped)
    with pytest.raises(AssertionError):
        PLT.test_cheb_eval_matches_plain()


def test_baby_rotation_without_the_p_lift_fails_its_pin(monkeypatch):
    """the double-hoisted baby rotation adding automorph(c0) without the factor P: the BSGS
    pin against the plain HMatmul fails"""
    from tests import test_oracle_plain as PLT
    monkeypatch.setattr(Oracle, "lift_p", lambda self, acc, x, level: _lift_unscaled(self, acc, x, level))
    o = Oracle(PP.Params(9, 6, 3, 60, 40, 60, h=32), 77)
    o.gen_relin_key()
    with pytest.raises(AssertionError):
        PLT.test_bsgs_double_hoisted_matches_plain(o)


def _lift_unscaled(self, acc, x, level):
    q = self.P.moduli(level)
    out = acc.copy()
    out[: level + 1] = C.add(acc[: level + 1], x, q)
    return out
