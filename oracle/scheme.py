"""RNS-CKKS scheme, fused CinS conv2d and bootstrapping steps of the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Ciphertexts are kept in the coefficient domain; products go through the NTT
(pinned to the schoolbook negacyclic product).  Every step follows the paper's
order (Alg. 1) and the standard hybrid RNS-CKKS the paper defers to (Sec. 2.1):

  key switching   digits of alpha consecutive limbs; ModUp by fast base conversion
                  without correction; inner product with the switching key over
                  Q_l u P; ModDown (c - Conv_{P->Q}([c]_P)) * P^{-1}.
  rotation        always "hoisted": ModUp(c1) once, then per rotation the Galois
                  automorphism on the raised digits, inner product, ModDown.
  HRot(ct, r)     slot j of the result holds slot j + r (Sec. 2.1), Galois 5^r.
  rescale         centred remainder of the last limb (Sec. 2.4).
  BSGS            sum_g rot_{a0+step*g*B}( sum_b d'_{g,b} (*) rot_{step*b}(ct) ),
                  d'_{g,b} = d_{a0+step(gB+b)} >> (a0+step*g*B)   (Sec. 2.5)

Scalar constants that become integers are rounded half away from zero from the
double products written next to them; the CUDA side forms the same products.
"""
import math

import numpy as np

from . import _clib as C
from . import encoding as E
from .params import (K_ENC_E0, K_ENC_E1, K_ENC_U, K_ENCSK_A, K_ENCSK_E, K_PK_A, K_PK_E,
                     K_SK, K_SK_SIGN, K_SWK_A, K_SWK_E, tag)


def round_half_away(x):
    """llround: nearest integer, halves away from zero."""
    return int(math.copysign(math.floor(abs(x) + 0.5), x))


class Ciphertext:
    def __init__(self, c0, c1, level, scale):
        self.c0 = np.ascontiguousarray(c0, dtype=np.uint64)
        self.c1 = np.ascontiguousarray(c1, dtype=np.uint64)
        self.level = level
        self.scale = float(scale)

    def copy(self):
        return Ciphertext(self.c0.copy(), self.c1.copy(), self.level, self.scale)


class Plaintext:
    def __init__(self, limbs, level, scale, ext=False):
        self.limbs = np.ascontiguousarray(limbs, dtype=np.uint64)   # coefficient domain
        self.level = level
        self.scale = float(scale)
        self.ext = ext          # limbs over Q_level u P (BSGS diagonals), else over Q_level


class BsgsPlan:
    """A linear map on the slots as BSGS over diagonals a0 + step*i, i < count.
    pts[(g, b)] is the pre-rotated diagonal plaintext (absent = zero diagonal)."""

    def __init__(self, a0, step, count, B, level, scale, pts):
        self.a0, self.step, self.count, self.B = a0, step, count, B
        self.level, self.scale = level, scale
        self.pts = pts

    @property
    def G(self):
        return -(-self.count // self.B)

    def rotations(self, m):
        """the rotation steps the plan's non-zero diagonals need (baby and giant)"""
        baby = [self.step * b % m for (_, b) in self.pts]
        giant = [(self.a0 + self.step * g * self.B) % m for (g, _) in self.pts]
        return sorted({r for r in baby + giant if r})


def power_in_y(c, alpha, beta):
    """sum_k c_k x^k with x = (y - beta) / alpha, as power coefficients in y (binomial expansion)"""
    out = [0.0] * len(c)
    for k, ck in enumerate(c):
        for j in range(k + 1):
            out[j] += ck * math.comb(k, j) * (-beta) ** (k - j) / alpha ** k
    return out


def default_bsgs_B(count):
    """Baby-step count: 2^ceil(log2(count)/2)."""
    return 1 << math.ceil(math.log2(count) / 2) if count > 1 else 1


def boot_bsgs_B(count):
    """Baby-step count for the bootstrapping HMatmuls: with double hoisting a baby step costs a
    key-switch inner product and a giant step about five times that (ModDown of c1, ModUp,
    inner product), so B minimises (B - 1) + 5 (G - 1), G = ceil(count / B), over powers of
    two (the smaller B on ties)."""
    best, bestB, B = None, 1, 1
    while True:
        G = -(-count // B)
        cost = (B - 1) + 5 * (G - 1)
        if best is None or cost < best:
            best, bestB = cost, B
        if B >= count:
            return bestB
        B *= 2


class Oracle:
    def __init__(self, params, seed):
        P = self.P = params
        self.seed = int(seed)
        n = P.n
        self.ops = {"pmult": 0, "hrot": 0, "keyswitch": 0, "hmult": 0, "rescale": 0, "modraise": 0}
        if P.h:
            s = C.sample_hw(n, P.h, self.seed, tag(K_SK), tag(K_SK_SIGN))
        else:
            s = C.sample_ternary(n, self.seed, tag(K_SK))
        self.s = s
        self.s_ntt = self.ntt(C.signed_to_rns(s, P.moduli(P.L, True)), P.L, True)
        qL = P.moduli(P.L)
        a = C.sample_uniform(qL, P.prime_ids(P.L), n, self.seed, tag(K_PK_A))
        e = self.ntt(C.signed_to_rns(C.sample_gauss(n, P.sigma, self.seed, tag(K_PK_E)), qL), P.L)
        b = C.sub(e, C.mul(a, self.s_ntt[: P.L + 1], qL), qL)
        self.pk = (b, a)
        self.swk = {}

    # ------------------------------------------------------------ helpers --
    def ext_rows(self, level):
        """rows of a full Q_L u P array that a level-`level` extended array uses"""
        return list(range(level + 1)) + [self.P.n_q + j for j in range(self.P.n_p)]

    def ntt(self, x, level, with_p=False):
        return C.ntt_forward(x, self.P.moduli(level, with_p), self.P.psis(level, with_p), self.P.logn)

    def intt(self, x, level, with_p=False):
        return C.ntt_inverse(x, self.P.moduli(level, with_p), self.P.psis(level, with_p), self.P.logn)

    def polymul(self, a, b, level):
        """negacyclic product of two coefficient-domain RNS polynomials"""
        q = self.P.moduli(level)
        return self.intt(C.mul(self.ntt(a, level), self.ntt(b, level), q), level)

    def galois(self, r):
        m = self.P.n // 2
        return pow(5, r % m, 2 * self.P.n)

    # -------------------------------------------------------------- keys ----
    def _gen_switch_key(self, code, sprime_ntt):
        """digit d: (b_d, a_d) with b_d = -a_d s + e_d + [P]_{q_i} s' on the digit's limbs."""
        P = self.P
        ext = P.moduli(P.L, True)
        ids = P.prime_ids(P.L, True)
        pmod = [1] * P.n_q
        for i in range(P.n_q):
            v = 1
            for pj in P.p:
                v = v * pj % P.q[i]
            pmod[i] = v
        kb, ka = [], []
        for d, limbs in enumerate(P.digits(P.L)):
            a = C.sample_uniform(ext, ids, P.n, self.seed, tag(K_SWK_A, code, d))
            e = C.sample_gauss(P.n, P.sigma, self.seed, tag(K_SWK_E, code, d))
            e = self.ntt(C.signed_to_rns(e, ext), P.L, True)
            b = C.sub(e, C.mul(a, self.s_ntt, ext), ext)
            for i in limbs:
                t = C.mul_scalar(sprime_ntt[i: i + 1], [pmod[i]], [P.q[i]])
                b[i] = C.add(b[i: i + 1], t, [P.q[i]])[0]
            kb.append(b)
            ka.append(a)
        self.swk[code] = (kb, ka)

    def gen_relin_key(self):
        ext = self.P.moduli(self.P.L, True)
        self._gen_switch_key(0, C.mul(self.s_ntt, self.s_ntt, ext))

    def gen_galois_key(self, g):
        P = self.P
        ext = P.moduli(P.L, True)
        sg = C.automorphism(C.signed_to_rns(self.s, ext), ext, g, P.logn)
        self._gen_switch_key(g, self.ntt(sg, P.L, True))

    def gen_rotation_keys(self, steps):
        for r in steps:
            g = self.galois(r)
            if g != 1 and g not in self.swk:
                self.gen_galois_key(g)

    def gen_conj_key(self):
        self.gen_galois_key(2 * self.P.n - 1)

    # ------------------------------------------------------- enc / dec ------
    def encode_pt(self, z, level, scale, ext=False):
        """slot vector z (N/2 complex) -> plaintext round(scale * f); ext: limbs over Q_level u P"""
        f = E.encode(z, self.P.n) * scale
        return self.pt_from_real_coeffs(f, level, scale, ext)

    def pt_from_real_coeffs(self, f, level, scale, ext=False):
        v = np.round(f)
        assert np.abs(v).max() < 2.0 ** 62, "plaintext coefficient too large"
        return Plaintext(C.signed_to_rns(v.astype(np.int64), self.P.moduli(level, ext)), level, scale, ext)

    def encrypt(self, pt, nonce):
        P, l, n = self.P, pt.level, self.P.n
        q = P.moduli(l)
        u = self.ntt(C.signed_to_rns(C.sample_ternary(n, self.seed, tag(K_ENC_U, nonce)), q), l)
        e0 = C.signed_to_rns(C.sample_gauss(n, P.sigma, self.seed, tag(K_ENC_E0, nonce)), q)
        e1 = C.signed_to_rns(C.sample_gauss(n, P.sigma, self.seed, tag(K_ENC_E1, nonce)), q)
        b, a = self.pk
        c0 = C.add(C.add(self.intt(C.mul(u, b[: l + 1], q), l), e0, q), pt.limbs, q)
        c1 = C.add(self.intt(C.mul(u, a[: l + 1], q), l), e1, q)
        return Ciphertext(c0, c1, l, pt.scale)

    def encrypt_sk(self, pt, nonce):
        P, l, n = self.P, pt.level, self.P.n
        q = P.moduli(l)
        a = C.sample_uniform(q, P.prime_ids(l), n, self.seed, tag(K_ENCSK_A, nonce))
        e = C.signed_to_rns(C.sample_gauss(n, P.sigma, self.seed, tag(K_ENCSK_E, nonce)), q)
        c0 = C.add(C.sub(e, self.intt(C.mul(a, self.s_ntt[: l + 1], q), l), q), pt.limbs, q)
        return Ciphertext(c0, self.intt(a, l), l, pt.scale)

    def decrypt(self, ct):
        l = ct.level
        q = self.P.moduli(l)
        m = C.add(ct.c0, self.intt(C.mul(self.ntt(ct.c1, l), self.s_ntt[: l + 1], q), l), q)
        return Plaintext(m, l, ct.scale)

    def centred_coeffs(self, pt):
        """exact centred integers of an RNS polynomial (CRT in Python integers), as floats"""
        q = self.P.moduli(pt.level)
        if len(q) == 1:
            v = pt.limbs[0].astype(np.int64)
            return np.where(v > q[0] // 2, v - np.int64(q[0]), v).astype(np.float64)
        Q = 1
        for x in q:
            Q *= x
        acc = np.zeros(pt.limbs.shape[1], dtype=object)
        for i, qi in enumerate(q):
            Qi = Q // qi
            inv = pow(Qi % qi, -1, qi)
            xi = pt.limbs[i].astype(object) * inv % qi
            acc = acc + xi * Qi
        acc = acc % Q
        acc = np.where(acc > Q // 2, acc - Q, acc)
        return np.array([float(v) for v in acc])

    def decode_slots(self, pt):
        return E.decode(self.centred_coeffs(pt) / pt.scale, self.P.n)

    def decode_coeffs(self, pt):
        return self.centred_coeffs(pt) / pt.scale

    # ------------------------------------------------------ arithmetic ------
    @staticmethod
    def _check_scales(a, b):
        assert a.level == b.level, (a.level, b.level)
        assert abs(a.scale - b.scale) <= 2.0 ** -30 * abs(a.scale), (a.scale, b.scale)

    def add(self, a, b):
        self._check_scales(a, b)
        q = self.P.moduli(a.level)
        return Ciphertext(C.add(a.c0, b.c0, q), C.add(a.c1, b.c1, q), a.level, a.scale)

    def sub(self, a, b):
        self._check_scales(a, b)
        q = self.P.moduli(a.level)
        return Ciphertext(C.sub(a.c0, b.c0, q), C.sub(a.c1, b.c1, q), a.level, a.scale)

    def mul_plain(self, ct, pt):
        """PMult without rescale"""
        assert pt.level == ct.level
        self.ops["pmult"] += 1
        l = ct.level
        q = self.P.moduli(l)
        p = self.ntt(pt.limbs, l)
        c0 = self.intt(C.mul(self.ntt(ct.c0, l), p, q), l)
        c1 = self.intt(C.mul(self.ntt(ct.c1, l), p, q), l)
        return Ciphertext(c0, c1, l, ct.scale * pt.scale)

    def mul_int(self, ct, c):
        """multiply by an integer constant c (|c| < 2^63); scale unchanged"""
        q = self.P.moduli(ct.level)
        r = [C.signed_to_rns(np.array([c], dtype=np.int64), [x])[0, 0] for x in q]
        return Ciphertext(C.mul_scalar(ct.c0, r, q), C.mul_scalar(ct.c1, r, q), ct.level, ct.scale)

    def add_const(self, ct, c):
        """add the real constant c to every slot: c0 += llround(c * scale) * X^0"""
        v = round_half_away(c * ct.scale)
        q = self.P.moduli(ct.level)
        c0 = ct.c0.copy()
        for i, qi in enumerate(q):
            c0[i, 0] = (int(c0[i, 0]) + v) % qi
        return Ciphertext(c0, ct.c1.copy(), ct.level, ct.scale)

    def imult(self, ct):
        """multiply every slot by i: polynomial times X^{N/2}"""
        q = self.P.moduli(ct.level)
        h = self.P.n // 2

        def shift(x):
            out = np.empty_like(x)
            out[:, h:] = x[:, :h]
            out[:, :h] = C.neg(np.ascontiguousarray(x[:, h:]), q)
            return out
        return Ciphertext(shift(ct.c0), shift(ct.c1), ct.level, ct.scale)

    def rescale(self, ct):
        self.ops["rescale"] += 1
        q = self.P.moduli(ct.level)
        return Ciphertext(C.rescale(ct.c0, q), C.rescale(ct.c1, q), ct.level - 1,
                          ct.scale / float(q[ct.level]))

    def mod_drop(self, ct, level):
        assert level <= ct.level
        return Ciphertext(ct.c0[: level + 1].copy(), ct.c1[: level + 1].copy(), level, ct.scale)

    def level_down(self, ct, level):
        """bring ct to `level` at the canonical scale: per level, multiply by the integer
        llround((Delta_{l-1} * q_l) / scale) and rescale"""
        P = self.P
        while ct.level > level:
            l = ct.level
            c = round_half_away((P.delta[l - 1] * float(P.q[l])) / ct.scale)
            ct = self.rescale(self.mul_int(ct, c))
            ct.scale = P.delta[l - 1]
        return ct

    def mod_raise(self, ct):
        assert ct.level == 0
        self.ops["modraise"] += 1
        q = self.P.moduli(self.P.L)
        return Ciphertext(C.mod_raise(ct.c0[0], q), C.mod_raise(ct.c1[0], q), self.P.L, ct.scale)

    # ------------------------------------------------------ key switching ----
    def mod_up(self, x, level):
        """per digit: [x]_{Q_d} raised to Q_l u P by fast base conversion"""
        P = self.P
        ext = P.moduli(level, True)
        out = []
        for limbs in P.digits(level):
            D = np.empty((len(ext), P.n), dtype=np.uint64)
            D[limbs] = x[limbs]
            others = [i for i in range(len(ext)) if i not in limbs]
            conv = C.base_convert(np.ascontiguousarray(x[limbs]), [ext[i] for i in limbs],
                                  [ext[i] for i in others])
            D[others] = conv
            out.append(D)
        return out

    def key_switch_inner(self, digits, code, level):
        """inner product of raised digits with switching key `code`: two polynomials over
        Q_l u P (coefficient domain), before ModDown"""
        P = self.P
        self.ops["keyswitch"] += 1
        ext = P.moduli(level, True)
        rows = self.ext_rows(level)
        kb, ka = self.swk[code]
        acc_b = np.zeros((len(ext), P.n), dtype=np.uint64)
        acc_a = np.zeros_like(acc_b)
        for d, D in enumerate(digits):
            Dn = self.ntt(D, level, True)
            C.mul_acc(acc_b, Dn, np.ascontiguousarray(kb[d][rows]), ext)
            C.mul_acc(acc_a, Dn, np.ascontiguousarray(ka[d][rows]), ext)
        return self.intt(acc_b, level, True), self.intt(acc_a, level, True)

    def key_switch_raised(self, digits, code, level):
        """inner product of raised digits with switching key `code`, then ModDown"""
        acc_b, acc_a = self.key_switch_inner(digits, code, level)
        q = self.P.moduli(level)
        return C.mod_down(acc_b, q, self.P.p), C.mod_down(acc_a, q, self.P.p)

    def lift_p(self, acc, x, level):
        """acc over Q_l u P plus P x (x over Q_l): rows 0..l += [P]_{q_i} x_i"""
        P = self.P
        q = P.moduli(level)
        pm = []
        for qi in q:
            v = 1
            for pj in P.p:
                v = v * (pj % qi) % qi
            pm.append(v)
        out = acc.copy()
        out[: level + 1] = C.add(acc[: level + 1], C.mul_scalar(x, pm, q), q)
        return out

    def mod_down_rescale(self, acc_b, acc_a, level):
        """ModDown fused with the rescale after it: the Q_l u P polynomials divided by M = q_l P
        with rounding, out_i = (a_i - r) M^{-1} mod q_i (i < l), r the centred remainder of a
        mod M.  Exact: r by the CRT written out in multi-precision integers."""
        P = self.P
        self.ops["rescale"] += 1
        S = [int(P.q[level])] + [int(x) for x in P.p]
        return self._div_round(acc_b, level, S), self._div_round(acc_a, level, S)

    def _div_round(self, acc, level, S):
        """acc rows q_0..q_l then the special primes (S = [q_l] + P) -> round(acc / prod S)"""
        return C.div_round(acc, level, self.P.moduli(level - 1), S)

    def rotate_hoisted(self, ct, steps):
        """HRot(ct, r) for every r in steps, sharing one ModUp of c1"""
        P = self.P
        l = ct.level
        q = P.moduli(l)
        ext = P.moduli(l, True)
        digits = None
        outs = []
        for r in steps:
            g = self.galois(r)
            if g == 1:
                outs.append(ct.copy())
                continue
            if digits is None:
                digits = self.mod_up(ct.c1, l)
            self.ops["hrot"] += 1
            dg = [C.automorphism(D, ext, g, P.logn) for D in digits]
            k0, k1 = self.key_switch_raised(dg, g, l)
            c0 = C.add(C.automorphism(ct.c0, q, g, P.logn), k0, q)
            outs.append(Ciphertext(c0, k1, l, ct.scale))
        return outs

    def rotate(self, ct, r):
        return self.rotate_hoisted(ct, [r])[0]

    def conjugate(self, ct):
        P = self.P
        l = ct.level
        q, ext = P.moduli(l), P.moduli(l, True)
        g = 2 * P.n - 1
        dg = [C.automorphism(D, ext, g, P.logn) for D in self.mod_up(ct.c1, l)]
        k0, k1 = self.key_switch_raised(dg, g, l)
        return Ciphertext(C.add(C.automorphism(ct.c0, q, g, P.logn), k0, q), k1, l, ct.scale)

    def mul_relin(self, a, b):
        """HMult with relinearisation, no rescale"""
        assert a.level == b.level
        self.ops["hmult"] += 1
        l = a.level
        q = self.P.moduli(l)
        a0, a1, b0, b1 = (self.ntt(x, l) for x in (a.c0, a.c1, b.c0, b.c1))
        d0 = self.intt(C.mul(a0, b0, q), l)
        d1 = self.intt(C.add(C.mul(a0, b1, q), C.mul(a1, b0, q), q), l)
        d2 = self.intt(C.mul(a1, b1, q), l)
        k0, k1 = self.key_switch_raised(self.mod_up(d2, l), 0, l)
        return Ciphertext(C.add(d0, k0, q), C.add(d1, k1, q), l, a.scale * b.scale)

    def mul_relin_rescale(self, a, b):
        """HMult, relinearisation and rescale, the relinearisation's ModDown fused with the
        rescale: (d0, d1) + keyswitch(d2) kept over Q_l u P and divided by P q_l at once"""
        assert a.level == b.level and a.level >= 1
        self.ops["hmult"] += 1
        l = a.level
        q = self.P.moduli(l)
        a0, a1, b0, b1 = (self.ntt(x, l) for x in (a.c0, a.c1, b.c0, b.c1))
        d0 = self.intt(C.mul(a0, b0, q), l)
        d1 = self.intt(C.add(C.mul(a0, b1, q), C.mul(a1, b0, q), q), l)
        d2 = self.intt(C.mul(a1, b1, q), l)
        kb, ka = self.key_switch_inner(self.mod_up(d2, l), 0, l)
        c0, c1 = self.mod_down_rescale(self.lift_p(kb, d0, l), self.lift_p(ka, d1, l), l)
        return Ciphertext(c0, c1, l - 1, a.scale * b.scale / float(self.P.q[l]))

    # ------------------------------------------------------------ BSGS -------
    def make_plan(self, diags, a0, step, count, level, scale, B=None):
        """diags: {offset: slot vector}; builds pre-rotated plaintexts d'_{g,b}"""
        m = self.P.n // 2
        B = B or default_bsgs_B(count)
        plan = BsgsPlan(a0 % m, step, count, B, level, scale, {})
        for g in range(plan.G):
            R = (plan.a0 + step * g * B) % m
            for b in range(B):
                i = g * B + b
                if i >= count:
                    break
                off = (plan.a0 + step * i) % m
                if off not in diags:
                    continue
                plan.pts[(g, b)] = self.encode_pt(np.roll(diags[off], R), level, scale, ext=True)
        return plan

    def bsgs(self, ct, plan, rescale=False):
        """sum_g rot_{a0+step*g*B}( sum_b pt_{g,b} (*) rot_{step*b}(ct) )"""
        return self.bsgs_multi([ct], [plan], rescale)

    def rotate_hoisted_ext(self, ct, steps):
        """rot_r(ct) for every r in steps, kept over Q_l u P before ModDown (double hoisting):
        (P automorph(c0) + u0, u1) with u the key switch of the automorphed ModUp digits of c1;
        r = 0 gives (P c0, P c1).  One ModUp of c1 serves all steps."""
        P = self.P
        l = ct.level
        q, ext = P.moduli(l), P.moduli(l, True)
        zeros = np.zeros((len(ext), P.n), dtype=np.uint64)
        digits = None
        outs = []
        for r in steps:
            g = self.galois(r)
            if g == 1:
                outs.append((self.lift_p(zeros, ct.c0, l), self.lift_p(zeros, ct.c1, l)))
                continue
            if digits is None:
                digits = self.mod_up(ct.c1, l)
            self.ops["hrot"] += 1
            dg = [C.automorphism(D, ext, g, P.logn) for D in digits]
            kb, ka = self.key_switch_inner(dg, g, l)
            outs.append((self.lift_p(kb, C.automorphism(ct.c0, q, g, P.logn), l), ka))
        return outs

    def bsgs_multi(self, cts, plans, rescale=False):
        """sum over inputs t and giant steps g of rot_{R_g}(sum_b pt_{g,b} (*) rot_{step b}(ct_t)),
        double hoisted: the baby-step rotations of each input share one ModUp and stay over
        Q_l u P (no ModDown), the plaintext diagonals are over Q_l u P, and the inner sums of
        all inputs with the same giant step are added there.  A giant step with R != 0 brings
        only its c1 down (ModDown), raises it (ModUp) and key-switches it; its c0 is
        automorphed over Q_l u P.  Everything is summed over Q_l u P and brought down once:
        ModDown, or ModDown fused with the rescale when `rescale` is set."""
        P = self.P
        l = cts[0].level
        m = P.n // 2
        q, ext = P.moduli(l), P.moduli(l, True)
        geo = {(p.a0, p.step, p.B, p.G) for p in plans}
        assert len(geo) == 1, "the plans of one HMatmul share their BSGS geometry"
        a0, step, B, G = geo.pop()
        inner = {}
        scale = None
        for ct, plan in zip(cts, plans):
            assert ct.level == plan.level == l
            used_b = sorted({b for (_, b) in plan.pts})
            babies = dict(zip(used_b, self.rotate_hoisted_ext(ct, [step * b % m for b in used_b])))
            bn = {b: (self.ntt(v[0], l, True), self.ntt(v[1], l, True)) for b, v in babies.items()}
            for (g, b), pt in plan.pts.items():
                assert pt.ext
                self.ops["pmult"] += 1
                pn = self.ntt(pt.limbs, l, True)
                t0, t1 = C.mul(bn[b][0], pn, ext), C.mul(bn[b][1], pn, ext)
                if g in inner:
                    inner[g] = (C.add(inner[g][0], t0, ext), C.add(inner[g][1], t1, ext))
                else:
                    inner[g] = (t0, t1)
                s_ = ct.scale * pt.scale
                assert scale is None or abs(s_ - scale) <= 1e-9 * scale
                scale = s_
        acc = None
        for g in sorted(inner):
            i0, i1 = self.intt(inner[g][0], l, True), self.intt(inner[g][1], l, True)
            R = (a0 + step * g * B) % m
            if R:
                gal = self.galois(R)
                self.ops["hrot"] += 1
                c1q = C.mod_down(i1, q, P.p)
                dg = [C.automorphism(D, ext, gal, P.logn) for D in self.mod_up(c1q, l)]
                kb, ka = self.key_switch_inner(dg, gal, l)
                i0, i1 = C.add(C.automorphism(i0, ext, gal, P.logn), kb, ext), ka
            acc = (i0, i1) if acc is None else (C.add(acc[0], i0, ext), C.add(acc[1], i1, ext))
        if rescale:
            c0, c1 = self.mod_down_rescale(acc[0], acc[1], l)
            return Ciphertext(c0, c1, l - 1, scale / float(P.q[l]))
        return Ciphertext(C.mod_down(acc[0], q, P.p), C.mod_down(acc[1], q, P.p), l, scale)

    # --------------------------------------------------- fused CinS conv ----
    def conv_plan(self, W, cin, cout, f, w, level, pt_scale, B=None):
        """Alg. 1, conv step: diagonals of S'K^ as a BSGS plan over offsets d*l, d < C"""
        n = self.P.n
        ell = w * w // 2
        C_ = n // (w * w)
        diags = E.fused_conv_diagonals(W, cin, cout, f, w, n)
        dd = {(d * ell) % (n // 2): diags[d] for d in range(C_) if np.abs(diags[d]).max() > 0}
        return self.make_plan(dd, 0, ell, C_, level, pt_scale, B)

    def conv2d_cins(self, ct, plan):
        return self.bsgs(ct, plan, rescale=True)

    def fc_plan(self, M, level, pt_scale, B=None):
        """FC fused with the whole StoC (Sec. 4.3): BSGS plan over the n_in diagonals of V M"""
        n_in = M.shape[1]
        return self.make_plan(E.fc_stoc_diagonals(M, self.P.n), 0, 1, n_in, level, pt_scale, B)

    def fc_replicate_steps(self, n_in):
        """rotations that replicate slots [0, n_in) over all N/2 slots: -n_in 2^t"""
        m = self.P.n // 2
        steps, s = [], n_in
        while s < m:
            steps.append((-s) % m)
            s *= 2
        return steps

    def fc_stoc(self, ct, plan, n_in):
        """x in slots [0, n_in), zero elsewhere -> replicate (x += rot(x, -n_in 2^t)) ->
        HMatmul(V M) -> rescale: the coefficients hold M x"""
        for r in self.fc_replicate_steps(n_in):
            ct = self.add(ct, self.rotate(ct, r))
        return self.bsgs(ct, plan, rescale=True)

    def dwconv_cins(self, ct, pt_kernel):
        """depthwise conv2d (Sec. 3.3.4): one PMult by the packed kernels, then rescale"""
        return self.rescale(self.mul_plain(ct, pt_kernel))

    # ------------------------------------------------------- bootstrapping ----
    # ------------------------------------------------ Chebyshev evaluation ----
    def prod_level(self, m):
        """level at which to multiply two ciphertexts available at level m: a product at the
        bottom level of the bootstrapping segment would not rescale onto the circuit
        segment's canonical scale, so it is taken one level lower"""
        P = self.P
        if P.n_boot > 0 and P.n_circuit >= 1 and m == P.n_circuit + 1:
            return m - 1
        return m

    def poly_out_level(self, level, depth):
        """level after `depth` multiplicative levels from `level` (one more if the segment
        boundary lies in between)"""
        P = self.P
        want = level - depth
        if P.n_boot > 0 and P.n_circuit >= 1 and want <= P.n_circuit < level:
            want -= 1
        return want

    def cheb_powers(self, x, ks):
        """T_k(x) for every k in ks (and what they need): T_k = 2 T_ceil(k/2) T_floor(k/2) -
        T_(k mod 2 ? 1 : 0), operands brought to a common level by level_down."""
        T = {1: x}
        cache = {}

        def at(k, lev):
            if T[k].level == lev:
                return T[k]
            if (k, lev) not in cache:
                cache[(k, lev)] = self.level_down(T[k], lev)
            return cache[(k, lev)]

        def need(k):
            if k in T:
                return
            a, b = k // 2, k - k // 2
            need(a)
            need(b)
            if a != b:
                need(b - a)
            m = self.prod_level(min(T[a].level, T[b].level))
            t = self.mul_relin_rescale(at(a, m), at(b, m))
            t = self.add(t, t)
            t = self.add_const(t, -1.0) if a == b else self.sub(t, at(b - a, m - 1))
            T[k] = t

        for k in sorted(ks):
            need(k)
        return T, at

    def cheb_leaf(self, T, at, coeffs):
        """sum_k c_k T_k for a low-degree piece.  The target level is the lowest level among
        its T_k minus one; every T_k is first brought to target + 1 by level_down (cached, so
        the leaves of one polynomial share it), multiplied by llround(c_k s_c) with
        s_c = Delta_target q_(target+1) / scale, summed and rescaled once.
        Returns a ciphertext, or a float when only the constant term is non-zero."""
        P = self.P
        ks = [k for k in range(1, len(coeffs)) if coeffs[k] != 0.0]
        if not ks:
            return float(coeffs[0])
        lev = min(T[k].level for k in ks)
        target = lev - 1
        acc = None
        for k in ks:
            t = at(k, lev)
            s_c = (P.delta[target] * float(P.q[lev])) / t.scale
            term = self.mul_int(t, round_half_away(coeffs[k] * s_c))
            if acc is None:
                acc = term
            else:
                acc = Ciphertext(C.add(acc.c0, term.c0, P.moduli(lev)), C.add(acc.c1, term.c1, P.moduli(lev)),
                                 lev, acc.scale)
        acc = self.rescale(acc)
        acc.scale = P.delta[target]
        return self.add_const(acc, coeffs[0])

    def cheb_eval(self, x, coeffs):
        """sum_k c_k T_k(x) by baby-step giant-step: baby steps T_1..T_b, giant steps
        T_b, T_2b, T_4b, ... (b = 2^ceil(m/2), m = ceil(log2(deg + 1))); the polynomial is split
        by Chebyshev division p = q T_n + r (n the largest giant <= deg; q_0 = c_n,
        q_j = 2 c_(n+j), r_(n-j) = c_(n-j) - c_(n+j)) down to pieces of degree < b, which are
        evaluated as leaves.  Depth ceil(log2 deg) + 1 for the degrees used here; the result
        is brought down to level(x) - ceil(log2 deg) - 1."""
        coeffs = [float(c) for c in coeffs]
        d = len(coeffs) - 1
        assert d >= 1
        m = math.ceil(math.log2(d + 1))
        b = 1 << ((m + 1) // 2)
        giants = []
        n = b
        while n <= d:
            giants.append(n)
            n *= 2
        T, at = self.cheb_powers(x, list(range(1, min(b, d + 1))) + giants)

        def rec(c):
            deg = len(c) - 1
            while deg > 0 and c[deg] == 0.0:
                deg -= 1
            c = c[: deg + 1]
            if deg < b:
                return self.cheb_leaf(T, at, c)
            n = max(g for g in giants if g <= deg)
            q = [c[n]] + [2.0 * c[n + j] for j in range(1, deg - n + 1)]
            r = list(c[:n])
            for j in range(1, deg - n + 1):
                r[n - j] -= c[n + j]
            Q, R = rec(q), rec(r)
            Tn = T[n]
            if isinstance(Q, float):
                if Q == 0.0:
                    prod = None
                else:
                    lk = Tn.level
                    s_c = (self.P.delta[lk - 1] * float(self.P.q[lk])) / Tn.scale
                    prod = self.rescale(self.mul_int(Tn, round_half_away(Q * s_c)))
                    prod.scale = (Tn.scale * s_c) / float(self.P.q[lk])
            else:
                lev = self.prod_level(min(Q.level, Tn.level))
                prod = self.mul_relin_rescale(self.level_down(Q, lev), at(n, lev))
            if isinstance(R, float):
                return R if prod is None else self.add_const(prod, R)
            if prod is None:
                return R
            lev = min(prod.level, R.level)
            return self.add(self.level_down(prod, lev), self.level_down(R, lev))

        out = rec(coeffs)
        assert not isinstance(out, float), "polynomial evaluates to a constant"
        depth = math.ceil(math.log2(d)) if d > 1 else 0
        want = self.poly_out_level(x.level, depth + 1)
        assert out.level >= want, (out.level, want)
        return self.level_down(out, want)

    def affine(self, x, alpha, beta):
        """alpha x + beta: x times the integer llround(alpha Delta_(l-1) q_l / scale), rescaled onto
        the canonical scale Delta_(l-1) (one level), then beta added"""
        P = self.P
        l = x.level
        assert l >= 1
        c = round_half_away(alpha * (P.delta[l - 1] * float(P.q[l])) / x.scale)
        y = self.rescale(self.mul_int(x, c))
        y.scale = P.delta[l - 1]
        return self.add_const(y, beta)

    def eval_poly(self, x, coeffs, a=-1.0, b=1.0, basis="cheb"):
        """p(x) for x in [a, b]: the variable y = (2x - a - b) / (b - a) by `affine` (skipped for
        [-1, 1]); a power-basis p is first re-expressed as a Chebyshev series in y (FP64: the
        binomial change of variable, then numpy's poly2cheb); then cheb_eval"""
        coeffs = [float(v) for v in coeffs]
        alpha, beta = 2.0 / (b - a), -(a + b) / (b - a)
        if basis == "power":
            coeffs = list(np.polynomial.chebyshev.poly2cheb(power_in_y(coeffs, alpha, beta)))
        y = x if (a == -1.0 and b == 1.0) else self.affine(x, alpha, beta)
        return self.cheb_eval(y, coeffs)

    def eval_mod(self, x, coeffs, r):
        """cos(2 pi (K y - 1/4) / 2^r) by Chebyshev, then r double angles -> sin(2 pi K y)"""
        y = self.cheb_eval(x, coeffs)
        for _ in range(r):
            y = self.mul_relin_rescale(y, y)
            y = self.add(y, y)
            y = self.add_const(y, -1.0)
        return y
