"""Alg. 1 block of the oracle: fused conv -> ModRaise -> CtoS -> EvalMod (Re, Im)
-> mask -> recombine -> StoC1.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings of the paper used here (it is silent on the bootstrapping internals and
defers them to the CKKS bootstrapping papers it cites in Sec. 2.4):

* After the fused conv the level-0 ciphertext holds t = Delta_0 o + q0 I in its
  coefficients.  ModRaise keeps that polynomial; its scale is declared
  q0 * K_eff so that the message is y = t / (q0 K_eff) in [-1, 1].
* Every HMatmul is a double-hoisted BSGS (Oracle.bsgs_multi); the bootstrapping plans take
  the baby-step count of boot_bsgs_B (16 for 63 diagonals).
* CtoS = T_{N/2}^{-1} (Sec. 2.4) in `ctos_levels` BSGS levels, largest stride first;
  every level's plaintexts are encoded at scale q_l, so the rescale keeps the
  scale; the 1/2 of the conjugate split is folded into the last level.
* Re = ct + conj(ct), Im = i (conj(ct) - ct) (Alg. 1, bootstrapping step), taken while the
  scale is still q0 K_eff so that the conjugation's key-switch noise is negligible.
* One integer multiply + rescale per part drops the scale to the canonical Delta
  of the next level (K_eff absorbs the rounding of that integer).
* EvalMod: Chebyshev interpolant of cos(2 pi (K_eff y - 1/4) / 2^r) of degree `deg`
  on [-1, 1], then r double-angle steps c <- 2c^2 - 1, giving sin(2 pi t / q0).
* Mask (Alg. 1, activation step): PMult by the 0/1 padding masks times q0 / (2 pi Delta_0),
  which also turns sin(2 pi t / q0) back into the conv output o.
* HActivation is not part of this block (it is evaluated by cheb_eval/eval_poly
  on its own).  Recombine Re + i Im, then HMatmul(S_{l<-1}) (StoC1) in
  `stoc_levels` BSGS levels at canonical scales (Alg. 1, StoC1 step).
* stride = 2 (the next conv downsamples, Alg. 2): between the recombination and the
  StoC1 the tail applies Alg. 2's decomposition (one HMatmul by the
  permutation sum_j (>> j l/4) calG_l (<< r_j), at canonical scale), and the StoC1 becomes
  S_{l/4<-1}: the output holds 4C polyphase slices of (w/2)^2 reals.
"""
import math

import numpy as np

from . import encoding as E
from .scheme import Oracle, boot_bsgs_B, round_half_away


class BootConfig:
    def __init__(self, orc: Oracle, w, w0, cout, K=28, r=3, deg=59, ctos_levels=3,
                 stoc_levels=3, delta0=2.0 ** 49, ctos_B=None, stoc_B=None, coeffs=None, stride=1,
                 decomp_B=None):
        P = orc.P
        n, m = P.n, P.n // 2
        self.w, self.w0, self.cout = w, w0, cout
        self.two_l = w * w
        self.ell = self.two_l // 2
        self.C = n // self.two_l
        self.K, self.r, self.deg = K, r, deg
        self.delta0 = float(delta0)
        L = P.L
        q0 = float(P.q[0])
        # --- ModRaise scale and the scale drop after CtoS
        self.l_drop = L - ctos_levels
        ld = self.l_drop
        self.c_drop = round_half_away((P.delta[ld - 1] * float(P.q[ld])) / (q0 * K))
        self.K_eff = (P.delta[ld - 1] * float(P.q[ld])) / (q0 * self.c_drop)
        self.s_raise = q0 * self.K_eff
        # --- CtoS plans
        self.ctos = []
        groups = E.ctos_groups(n, ctos_levels)
        for i, (D, strides) in enumerate(groups):
            if i == len(groups) - 1:
                D = {o: 0.5 * v for o, v in D.items()}
            a0, step, count = E.ap_of_group(strides, m)
            lev = L - i
            B = ctos_B[i] if ctos_B else boot_bsgs_B(count)
            self.ctos.append(orc.make_plan(D, a0, step, count, lev, float(P.q[lev]), B))
        # --- EvalMod polynomial
        if coeffs is None:
            Ke, rr = self.K_eff, r

            def f(y):
                return np.cos(2.0 * np.pi * (Ke * y - 0.25) / (2.0 ** rr))
            coeffs = np.polynomial.chebyshev.chebinterpolate(f, deg)
        self.coeffs = [float(c) for c in coeffs]
        depth = math.ceil(math.log2(deg)) if deg > 1 else 1
        self.l_em = (ld - 1) - (depth + 1) - r
        assert self.l_em - 1 - stoc_levels >= 0, "not enough levels for the block"
        # --- masks (times q0 / (2 pi Delta_0))
        # the EvalMod output (last double angle rescaled by q_{l_em+1}) has scale s_em; the
        # mask plaintext scale makes the masked ciphertext land on Delta_{l_em-1}
        le = self.l_em
        self.s_em = (P.delta[le + 1] * P.delta[le + 1]) / float(P.q[le + 1])
        self.s_mask = (P.delta[le - 1] * float(P.q[le])) / self.s_em
        self.mask_re, self.mask_im = self.mask_vectors(q0 / (2.0 * np.pi * self.delta0))
        self.pt_mask_re = orc.encode_pt(self.mask_re, le, self.s_mask)
        self.pt_mask_im = orc.encode_pt(self.mask_im, le, self.s_mask)
        # --- stride 2: the Alg. 2 decomposition, then StoC1 over slices of l/4
        assert stride in (1, 2)
        self.stride = stride
        self.decomp = None
        top, ell_out = self.l_em - 1, self.ell
        if stride == 2:
            assert w >= 4 and w0 % 2 == 0
            a0, step, count = E.decompose_ap(w, n)
            self.decomp = orc.make_plan(E.decompose_diag(w, n), a0, step, count, top, P.delta[top],
                                        decomp_B if decomp_B else boot_bsgs_B(count))
            top, ell_out = top - 1, self.ell // 4
        # --- StoC1 plans
        self.stoc = []
        for i, (D, strides) in enumerate(E.stoc1_groups(n, ell_out, stoc_levels)):
            a0, step, count = E.ap_of_group(strides, m)
            lev = top - i
            B = stoc_B[i] if stoc_B else boot_bsgs_B(count)
            self.stoc.append(orc.make_plan(D, a0, step, count, lev, P.delta[lev], B))
        self.l_out = top - len(self.stoc)
        assert self.l_out >= 1, "not enough levels for the block"

    def mask_vectors(self, value):
        """slot i*l + u carries pixel rev_l(u) (Re) or rev_l(u) + l (Im) of output channel i;
        1 where that pixel is inside the w0 x w0 image of a real channel, else 0."""
        ell, w, w0 = self.ell, self.w, self.w0
        rev = E.bitrev_indices(ell)
        re = np.zeros(self.C * ell)
        im = np.zeros(self.C * ell)
        for i in range(self.cout):
            for u in range(ell):
                k = rev[u]
                for pix, vec in ((k, re), (k + ell, im)):
                    if pix // w < w0 and pix % w < w0:
                        vec[i * ell + u] = value
        return re, im


def mod_raise(orc: Oracle, ct0, cfg: BootConfig):
    """ModRaise, the result declared at scale q0 K_eff"""
    x = orc.mod_raise(ct0)
    x.scale = cfg.s_raise
    return x


def conj_split(orc: Oracle, x, cfg: BootConfig):
    """Re = x + conj(x), Im = i (conj(x) - x), each brought to the canonical scale by one
    integer multiply and rescale"""
    P = orc.P
    cj = orc.conjugate(x)
    re = orc.add(x, cj)
    im = orc.imult(orc.sub(cj, x))
    re = orc.rescale(orc.mul_int(re, cfg.c_drop))
    im = orc.rescale(orc.mul_int(im, cfg.c_drop))
    re.scale = P.delta[re.level]
    im.scale = P.delta[im.level]
    return re, im


def mask_recombine(orc: Oracle, re, im, cfg: BootConfig):
    """mask both parts, Re + i Im, and the Alg. 2 decomposition of a stride-2 block"""
    a = orc.rescale(orc.mul_plain(re, cfg.pt_mask_re))
    b = orc.rescale(orc.mul_plain(im, cfg.pt_mask_im))
    y = orc.add(a, orc.imult(b))
    if cfg.decomp is not None:
        y = orc.bsgs(y, cfg.decomp, rescale=True)
    return y


def bootstrap(orc: Oracle, ct0, cfg: BootConfig):
    """ModRaise -> CtoS -> scale drop -> conjugate split -> EvalMod (Re), EvalMod (Im)"""
    x = mod_raise(orc, ct0, cfg)
    for plan in cfg.ctos:
        x = orc.bsgs(x, plan, rescale=True)
    re, im = conj_split(orc, x, cfg)
    re = orc.eval_mod(re, cfg.coeffs, cfg.r)
    im = orc.eval_mod(im, cfg.coeffs, cfg.r)
    return re, im


def stoc1(orc: Oracle, re, im, cfg: BootConfig):
    """mask, Re + i Im, HMatmul(S_{l<-1})"""
    y = mask_recombine(orc, re, im, cfg)
    for plan in cfg.stoc:
        y = orc.bsgs(y, plan, rescale=True)
    return y


def block(orc: Oracle, ct_in, conv_plan, cfg: BootConfig):
    """One conv2d + bootstrap block (Alg. 1 without HActivation)."""
    x = orc.conv2d_cins(ct_in, conv_plan)
    assert abs(x.scale - cfg.delta0) <= 1e-9 * cfg.delta0
    re, im = bootstrap(orc, x, cfg)
    return stoc1(orc, re, im, cfg)


def block_stages(orc: Oracle, conv_plan, cfg: BootConfig):
    """The block's steps in order, as (name, step) pairs: each step takes the list of
    ciphertexts the previous one returned (first [ct_in]) and returns the next list; chained
    they compute block().  Used to time a block one step at a time."""
    def conv(v):
        x = orc.conv2d_cins(v[0], conv_plan)
        assert abs(x.scale - cfg.delta0) <= 1e-9 * cfg.delta0
        return [x]
    stages = [("conv", conv),
              ("modraise_ctos0", lambda v: [orc.bsgs(mod_raise(orc, v[0], cfg), cfg.ctos[0], rescale=True)])]
    for i, plan in enumerate(cfg.ctos[1:], 1):
        stages.append(("ctos%d" % i, lambda v, p=plan: [orc.bsgs(v[0], p, rescale=True)]))
    stages.append(("conj_split", lambda v: list(conj_split(orc, v[0], cfg))))
    stages.append(("evalmod_re", lambda v: [orc.eval_mod(v[0], cfg.coeffs, cfg.r), v[1]]))
    stages.append(("evalmod_im", lambda v: [v[0], orc.eval_mod(v[1], cfg.coeffs, cfg.r)]))
    stages.append(("mask_recombine", lambda v: [mask_recombine(orc, v[0], v[1], cfg)]))
    for i, plan in enumerate(cfg.stoc):
        stages.append(("stoc%d" % i, lambda v, p=plan: [orc.bsgs(v[0], p, rescale=True)]))
    return stages


def block_multi(orc: Oracle, cts, conv_plans, cfg: BootConfig):
    """conv2d over several input ciphertexts, then bootstrap + StoC1 tail.  With the
    decomposed kernels of a stride-2 conv this is Alg. 2 from the decomposed convs to the end
    (BSGS per input ciphertext, HAdd, one rescale; the giant steps of both share one ModDown fused with the
    rescale); with plain kernels it is the C_in > C generalisation
    (Sec. 3.3.3: the block matrix-vector product, one output ciphertext)."""
    x = orc.bsgs_multi(cts, conv_plans, rescale=True)
    assert abs(x.scale - cfg.delta0) <= 1e-9 * cfg.delta0
    re, im = bootstrap(orc, x, cfg)
    return stoc1(orc, re, im, cfg)


def block_rotations(orc: Oracle, conv_plan, cfg: BootConfig):
    m = orc.P.n // 2
    rots = set(conv_plan.rotations(m)) if conv_plan is not None else set()
    extra = [cfg.decomp] if cfg.decomp is not None else []
    for p in cfg.ctos + cfg.stoc + extra:
        rots |= set(p.rotations(m))
    return sorted(rots)
