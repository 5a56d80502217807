"""The plain, unfused forms of the oracle's restructured steps.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The scheme module takes three standard restructurings of the RNS-CKKS key switch
that the paper leaves open (Sec. 2.1 defers the scheme to RNS-CKKS):
  * double-hoisted BSGS: baby rotations kept over Q_l u P, one ModDown per HMatmul;
  * ModDown fused with the rescale that follows it: one rounded division by P q_l;
  * Chebyshev evaluation by baby steps, giant steps and Chebyshev division.
This module states the same operations without any of them, step by step as the
textbook scheme writes them, so that the restructured forms can be checked against
them (tests/test_oracle_plain.py):
  * every rotation is its own key switch with its own ModDown (Sec. 2.1, HRot);
  * a product is HMult, relinearisation with ModDown, then a separate rescale (Sec. 2.4);
  * an HMatmul is sum_g rot_{R_g}(sum_b pt_{g,b} (*) rot_{step b}(ct)) (Sec. 2.5, Eq. 3),
    with each plaintext multiplied over Q_l only;
  * a Chebyshev series is sum_k c_k T_k with every T_k from the product rule
    T_{a+b} = 2 T_a T_b - T_{|a-b|} (a = floor(k/2), b = ceil(k/2)), no division.
The results are not bit-identical to the restructured forms (their roundings differ
by a few units); they agree within the key-switch and rescale rounding bounds the
tests derive.
"""
import math

import numpy as np

from . import _clib as C
from .scheme import Ciphertext, Plaintext, round_half_away


def q_part(pt):
    """a plaintext over Q_l u P restricted to its Q_l rows (the same integers mod q_i)"""
    if not pt.ext:
        return pt
    return Plaintext(pt.limbs[: pt.level + 1].copy(), pt.level, pt.scale, ext=False)


def mul_relin_then_rescale(o, a, b):
    """HMult with relinearisation (its own ModDown), then a separate rescale"""
    return o.rescale(o.mul_relin(a, b))


def bsgs(o, cts, plans, rescale=False):
    """sum over inputs t and giant steps g of rot_{R_g}(sum_b pt_{g,b} (*) rot_{step b}(ct_t)):
    each baby and giant rotation a separate HRot (ModUp, key switch, ModDown), each
    product a PMult over Q_l, then one rescale when `rescale` is set"""
    m = o.P.n // 2
    acc = None
    geo = {(p.a0, p.step, p.B, p.G) for p in plans}
    assert len(geo) == 1
    a0, step, B, G = geo.pop()
    for g in range(G):
        inner = None
        for ct, plan in zip(cts, plans):
            for b in range(B):
                pt = plan.pts.get((g, b))
                if pt is None:
                    continue
                rb = step * b % m
                baby = o.rotate(ct, rb) if rb else ct
                t = o.mul_plain(baby, q_part(pt))
                inner = t if inner is None else o.add(inner, t)
        if inner is None:
            continue
        R = (a0 + step * g * B) % m
        giant = o.rotate(inner, R) if R else inner
        acc = giant if acc is None else o.add(acc, giant)
    return o.rescale(acc) if rescale else acc


def cheb_powers(o, x, kmax):
    """T_1..T_kmax by T_{a+b} = 2 T_a T_b - T_{|a-b|}, a = floor(k/2), b = ceil(k/2)
    (T_0 = 1: the constant -1 when a = b); operands brought to a common level by
    level_down, products at the oracle's product level (the segment boundary rule)."""
    T = {1: x}
    for k in range(2, kmax + 1):
        a, b = k // 2, k - k // 2
        lev = o.prod_level(min(T[a].level, T[b].level))
        t = mul_relin_then_rescale(o, o.level_down(T[a], lev), o.level_down(T[b], lev))
        t = o.add(t, t)
        if a == b:
            t = o.add_const(t, -1.0)
        else:
            t = o.sub(t, o.level_down(T[b - a], t.level))
        T[k] = t
    return T


def cheb_eval(o, x, coeffs):
    """sum_k c_k T_k(x) term by term: every T_k with c_k != 0 brought to one level lev (the
    lowest among them), multiplied by the integer llround(c_k s_c) with
    s_c = Delta_(lev-1) q_lev / scale, summed, rescaled once, c_0 added; then brought to
    the level the polynomial's depth leaves, level(x) - ceil(log2 deg) - 1"""
    P = o.P
    coeffs = [float(c) for c in coeffs]
    d = len(coeffs) - 1
    ks = [k for k in range(1, d + 1) if coeffs[k] != 0.0]
    assert ks, "polynomial evaluates to a constant"
    T = cheb_powers(o, x, max(ks))
    lev = min(T[k].level for k in ks)
    acc = None
    for k in ks:
        t = o.level_down(T[k], lev)
        s_c = (P.delta[lev - 1] * float(P.q[lev])) / t.scale
        term = o.mul_int(t, round_half_away(coeffs[k] * s_c))
        acc = term if acc is None else Ciphertext(C.add(acc.c0, term.c0, P.moduli(lev)),
                                                  C.add(acc.c1, term.c1, P.moduli(lev)), lev, acc.scale)
    acc = o.rescale(acc)
    acc.scale = P.delta[lev - 1]
    acc = o.add_const(acc, coeffs[0])
    depth = math.ceil(math.log2(d)) if d > 1 else 0
    want = o.poly_out_level(x.level, depth + 1)
    assert acc.level >= want, (acc.level, want)
    return o.level_down(acc, want)


def eval_mod(o, x, coeffs, r):
    """Chebyshev series of the shifted cosine, then r double angles y <- 2 y^2 - 1"""
    y = cheb_eval(o, x, coeffs)
    for _ in range(r):
        y = mul_relin_then_rescale(o, y, y)
        y = o.add(y, y)
        y = o.add_const(y, -1.0)
    return y


def bootstrap(o, ct0, cfg):
    """ModRaise -> CtoS -> conjugate split -> scale drop -> EvalMod (Re), EvalMod (Im), the
    same steps as oracle.boot.bootstrap with every HMatmul and product in its plain form"""
    P = o.P
    x = o.mod_raise(ct0)
    x.scale = cfg.s_raise
    for plan in cfg.ctos:
        x = bsgs(o, [x], [plan], rescale=True)
    cj = o.conjugate(x)
    re = o.add(x, cj)
    im = o.imult(o.sub(cj, x))
    re = o.rescale(o.mul_int(re, cfg.c_drop))
    im = o.rescale(o.mul_int(im, cfg.c_drop))
    re.scale = P.delta[re.level]
    im.scale = P.delta[im.level]
    return eval_mod(o, re, cfg.coeffs, cfg.r), eval_mod(o, im, cfg.coeffs, cfg.r)


def stoc1(o, re, im, cfg):
    """mask, Re + i Im, [Alg. 2 decomposition], HMatmul(S_{l<-1}) levels"""
    a = o.rescale(o.mul_plain(re, cfg.pt_mask_re))
    b = o.rescale(o.mul_plain(im, cfg.pt_mask_im))
    y = o.add(a, o.imult(b))
    if cfg.decomp is not None:
        y = bsgs(o, [y], [cfg.decomp], rescale=True)
    for plan in cfg.stoc:
        y = bsgs(o, [y], [plan], rescale=True)
    return y


def block(o, ct_in, conv_plan, cfg):
    """Alg. 1 without HActivation, every step in its plain form"""
    x = bsgs(o, [ct_in], [conv_plan], rescale=True)
    re, im = bootstrap(o, x, cfg)
    return stoc1(o, re, im, cfg)
