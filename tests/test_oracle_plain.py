"""Pins of the oracle's restructured key-switch steps.

The scheme module fuses three steps the paper leaves to RNS-CKKS (Sec. 2.1): the ModDown of
a key switch with the rescale after it (one rounded division by P q_l, Sec. 2.4), the BSGS
baby rotations kept over Q_l u P with one ModDown per HMatmul (Sec. 2.5), and the
Chebyshev evaluation by baby steps, giant steps and Chebyshev division.  Each is checked
here against a statement that does not use it:

* the fused division against round(X / (q_l P)) in Python integers;
* the fused HMult + rescale against HMult, ModDown and rescale done one after the other
  (within one unit per coefficient, the bound of two roundings of nearby reals);
* the double-hoisted BSGS and the Chebyshev evaluation against the plain forms of
  oracle/plain.py, within error bounds derived from the key-switch rounding;
* the whole Alg. 1 block against its plain form.
"""
import math
import random

import numpy as np
import pytest

from oracle import boot as BT
from oracle import encoding as E
from oracle import params as PP
from oracle import plain as PL
from oracle.scheme import Ciphertext, Oracle, Plaintext

rng = np.random.default_rng(23)


def _residues(x, moduli):
    return np.array([[v % m for v in x] for m in moduli], dtype=np.uint64)


def _crt_centred(rows, moduli):
    """exact centred integers of RNS rows (Python ints)"""
    M = math.prod(int(m) for m in moduli)
    out = []
    for j in range(rows.shape[1]):
        v = 0
        for i, m in enumerate(moduli):
            Mi = M // int(m)
            v += int(rows[i, j]) * pow(Mi % int(m), -1, int(m)) * Mi
        v %= M
        out.append(v - M if v > M // 2 else v)
    return out


@pytest.mark.parametrize("level", [1, 3])
def test_mod_down_rescale_is_rounded_division(level):
    """Oracle.mod_down_rescale on X over Q_l u P gives round(X / (q_l P)) mod Q_{l-1} on both
    polynomials: the exact rounded division of Sec. 2.4's rescale composed with the ModDown
    division by P (no tie can occur: q_l P is odd)"""
    P = PP.Params(4, 4, 2, 60, 40, 60, n_p=2)
    o = Oracle(P, 1)
    q = [int(v) for v in P.q[: level + 1]]
    p = [int(v) for v in P.p]
    QP = math.prod(q) * math.prod(p)
    M = q[level] * math.prod(p)
    n = P.n
    xs = [[random.randrange(QP) for _ in range(n)] for _ in range(2)]
    # the largest and smallest residues mod M, and values next to the rounding boundary
    xs[0][:4] = [0, QP - 1, M // 2, M // 2 + 1]
    acc = [_residues(x, q + p) for x in xs]
    outs = o.mod_down_rescale(acc[0], acc[1], level)
    for x, out in zip(xs, outs):
        assert out.shape == (level, n)
        for j in range(n):
            want = (2 * x[j] + M) // (2 * M)          # floor(X / M + 1/2)
            assert abs(want * M - x[j]) <= M // 2
            for i in range(level):
                assert int(out[i, j]) == want % q[i], (i, j)


@pytest.fixture(scope="module")
def small():
    P = PP.Params(9, 6, 3, 60, 40, 60, h=32)
    o = Oracle(P, 77)
    o.gen_relin_key()
    o.gen_conj_key()
    return o


def _slots(o, ct):
    return o.decode_slots(o.decrypt(ct))


def test_fused_product_within_one_unit_of_two_step(small):
    """HMult + relinearisation + rescale with the ModDown fused into the rescale against HMult,
    ModDown, rescale in sequence: the two-step form rounds Y / q_l with Y = (A - rho) / P,
    rho = A mod P + u P (0 <= u < n_p), the fused form rounds A / (P q_l); the two reals differ
    by rho / (P q_l) < n_p / q_l, so the results differ by at most one unit per coefficient,
    and only where a half-integer falls between them (probability below n_p / q_l ~ 2^-39 per
    coefficient): on these seeded inputs they are identical"""
    o = small
    L = o.P.L
    m = o.P.n // 2
    za = rng.normal(size=m) + 1j * rng.normal(size=m)
    zb = rng.normal(size=m) + 1j * rng.normal(size=m)
    for lev in (L, 2):
        a = o.encrypt(o.encode_pt(za, lev, o.P.delta[lev]), 1)
        b = o.encrypt(o.encode_pt(zb, lev, o.P.delta[lev]), 2)
        fused = o.mul_relin_rescale(a, b)
        two = PL.mul_relin_then_rescale(o, a, b)
        assert fused.level == two.level == lev - 1
        assert abs(fused.scale - two.scale) <= 1e-12 * two.scale
        q = o.P.moduli(lev - 1)
        for f, t in ((fused.c0, two.c0), (fused.c1, two.c1)):
            d = _crt_centred(np.array([(f[i].astype(object) - t[i].astype(object)) % int(qi)
                                       for i, qi in enumerate(q)], dtype=np.uint64), q)
            assert max(abs(v) for v in d) <= 1
            assert not any(d)
        assert np.abs(_slots(o, fused) - za * zb).max() < 1e-5


def _ks_bound(o, count, dmax):
    """decoded error, in the slots, that per-rotation ModDown rounding can add to an HMatmul
    of `count` diagonals with |d| <= dmax: each rounded polynomial is off by less than n_p
    per coefficient on c0 and c1, so the decryption is off by n_p (1 + ||s||_1) per
    coefficient, at most N n_p (1 + ||s||_1) in the canonical embedding; the plaintext
    multiplies it by at most dmax (its scale q_l is divided out by the rescale); each baby
    and giant rotation contributes one such term"""
    P = o.P
    s1 = int(np.abs(o.s).sum())
    per = P.n * P.n_p * (1 + s1)
    return (count * dmax + count) * per


def test_bsgs_double_hoisted_matches_plain(small):
    """Oracle.bsgs (double hoisted, one ModDown fused with the rescale per HMatmul) and the plain
    HMatmul (a key switch and ModDown per rotation, PMult over Q_l, separate rescale) decode to
    the same slots within the rounding bound, and both to the FP64 matrix product"""
    o = small
    P = o.P
    m = P.n // 2
    L = P.L
    a0, step, count, B = 5, 3, 21, 4
    diags = {(a0 + step * i) % m: 0.4 * (rng.normal(size=m) + 1j * rng.normal(size=m)) for i in range(count)}
    z = rng.normal(size=m) + 1j * rng.normal(size=m)
    ct = o.encrypt(o.encode_pt(z, L, P.delta[L]), 5)
    plan = o.make_plan(diags, a0, step, count, L, float(P.q[L]), B)
    o.gen_rotation_keys(plan.rotations(m))
    fused = o.bsgs(ct, plan, rescale=True)
    plain = PL.bsgs(o, [ct], [plan], rescale=True)
    assert fused.level == plain.level == L - 1
    want = E.diag_apply(diags, z)
    gf, gp = _slots(o, fused), _slots(o, plain)
    dmax = max(np.abs(v).max() for v in diags.values())
    bound = _ks_bound(o, count, dmax) / P.delta[L - 1] + 1e-9
    assert np.abs(gf - gp).max() <= bound, (np.abs(gf - gp).max(), bound)
    assert np.abs(gf - want).max() < 1e-5 and np.abs(gp - want).max() < 1e-5


def _cheb_bound(o, coeffs, x_level, e_in):
    """error bound of sum c_k T_k(x) for |x| <= 1 given input noise e_in: T_{a+b} =
    2 T_a T_b - T_{|a-b|} with |T| <= 1 adds 2 (e_a + e_b) + e_{|a-b|} plus one product's
    rounding (key switch and rescale: N (n_p + 2) (1 + ||s||_1) / Delta at its level) and a
    level_down's rounding per operand; the series adds sum |c_k| e_k and its own rounding"""
    P = o.P
    s1 = int(np.abs(o.s).sum())
    depth = math.ceil(math.log2(len(coeffs) - 1)) + 1
    step = P.n * (P.n_p + 2) * (1 + s1) / min(P.delta[max(1, x_level - depth - 1): x_level + 1])
    e = {1: e_in}
    for k in range(2, len(coeffs)):
        a, b = k // 2, k - k // 2
        e[k] = 2 * (e[a] + e[b]) + (e[b - a] if b != a else 0.0) + 4 * step
    return sum(abs(c) * e[k] for k, c in enumerate(coeffs) if k) + 4 * step * (len(coeffs) + 1)


def test_cheb_eval_matches_plain():
    """the EvalMod Chebyshev series of the config-2 chain (degree 59, N = 2^10) by BSGS with
    Chebyshev division and by the plain term-by-term series: both decode to the FP64 series
    within the derived noise bound, and they end on the same level and scale"""
    from tests.pairs import oracle_params
    P = oracle_params("cfg2_small")
    o = Oracle(P, 12)
    o.gen_relin_key()
    cfg = BT.BootConfig(o, 8, 4, 4)
    lev = cfg.l_drop - 1
    m = P.n // 2
    y = rng.uniform(-1, 1, m)
    ct = o.encrypt(o.encode_pt(y, lev, P.delta[lev]), 3)
    fused = o.cheb_eval(ct, cfg.coeffs)
    plain = PL.cheb_eval(o, ct, cfg.coeffs)
    assert fused.level == plain.level
    assert abs(fused.scale - plain.scale) <= 1e-12 * fused.scale
    want = np.polynomial.chebyshev.chebval(y, cfg.coeffs)
    e_in = np.abs(_slots(o, ct) - y).max()
    bound = _cheb_bound(o, cfg.coeffs, lev, e_in)
    ef = np.abs(_slots(o, fused).real - want).max()
    ep = np.abs(_slots(o, plain).real - want).max()
    assert ef <= bound and ep <= bound, (ef, ep, bound)
    # tight enough that dropping or flipping the sign of any of the 34 terms with |c_k| > 2^-15
    # (every k <= 34 here) takes the result outside it
    assert bound < 2.0 ** -16
    assert np.abs(_slots(o, fused) - _slots(o, plain)).max() <= 2 * bound


@pytest.mark.slow
def test_block_matches_plain():
    """Alg. 1 block at N = 2^10 on the config-2 chain: the oracle's restructured block and the
    plain block (every rotation its own ModDown, separate rescales, term-by-term Chebyshev)
    end on the same level and scale and both decode to the masked FP64 conv within 2^-12"""
    P = PP.Params(10, 24, 3, 60, 42, 60, h=192, n_p=7, boot_bits=48, n_boot=14)
    o = Oracle(P, 9)
    w0, w, f = 4, 8, 3
    C = P.n // (w * w)
    cin = cout = 4
    x = rng.random((cin, w0, w0))
    W = rng.normal(0, 0.1, (cout, cin, f, f))
    ct = o.encrypt(o.encode_pt(E.cins_input_slots(x, w, P.n), 1, P.delta[1]), 3)
    cfg = BT.BootConfig(o, w, w0, cout)
    plan = o.conv_plan(W, cin, cout, f, w, 1, (cfg.delta0 * float(P.q[1])) / ct.scale)
    o.gen_rotation_keys(BT.block_rotations(o, plan, cfg))
    o.gen_conj_key()
    o.gen_relin_key()
    fused = BT.block(o, ct, plan, cfg)
    plain = PL.block(o, ct, plan, cfg)
    assert fused.level == plain.level == cfg.l_out
    assert abs(fused.scale - plain.scale) <= 1e-12 * fused.scale
    ell = w * w // 2
    conv = E.conv2d_same(x, W)
    ref = np.zeros((C, w * w))
    for i in range(cout):
        ref[i] = E.flatten_padded(conv[i], w)
    for out in (fused, plain):
        got = _slots(o, out)
        pix = np.stack([E.encode(got[i * ell:(i + 1) * ell], w * w) for i in range(C)])
        assert np.abs(pix - ref).max() < 2.0 ** -12
