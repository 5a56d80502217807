"""Helpers for the parity tests: the same parameters and seed on both sides.

The oracle (CPU) and the CUDA library share only the seeded inputs of workloads.py;
everything else is computed independently and compared here.
"""
import numpy as np

import workloads as WL
from oracle import params as PP
from oracle.scheme import Oracle, Plaintext


def oracle_params(name):
    d = WL.PARAMS[name]
    return PP.Params(d["log_n"], d["n_q"], d["dnum"], d["q0_bits"], d["scale_bits"], d["p_bits"], h=d["h"],
                     sigma=d["sigma"], n_p=d["n_p"] or None, boot_bits=d["boot_bits"], n_boot=d["n_boot"])


def gpu_ctx(name, seed):
    import torch

    from paper_2312_04356_gb300 import ckks as K
    return K.ckks_ctx_create(WL.PARAMS[name], seed, torch.cuda.current_stream().cuda_stream)


def ct_limbs(ct):
    """oracle ciphertext -> [2][l+1][N] coefficient-domain limbs"""
    return np.stack([ct.c0, ct.c1])


def import_ct(K, ctx, ct):
    return K.ckks_ct_import_rns(ctx, ct_limbs(ct), ct.level, ct.scale)


def import_pt(K, ctx, pt: Plaintext):
    return K.ckks_pt_import_rns(ctx, pt.limbs, pt.level, pt.scale)


def import_plan(K, ctx, plan):
    ps = K.ckks_ptset_create(ctx, plan.a0, plan.step, plan.count, plan.B, plan.level, plan.scale)
    for (g, b), pt in plan.pts.items():
        K.ckks_ptset_set_rns(ctx, ps, g, b, pt.limbs)
    return ps


def assert_ct_equal(K, ctx, gct, oct_, what=""):
    got = K.ckks_ct_export_rns(ctx, gct)
    want = ct_limbs(oct_)
    lev, sc = K.ckks_ct_info(gct)
    assert lev == oct_.level, "%s: level %d != %d" % (what, lev, oct_.level)
    assert got.shape == want.shape, what
    bad = np.argwhere(got != want)
    assert bad.size == 0, "%s: %d limb words differ, first at %s" % (what, len(bad), bad[:3].tolist())
    assert abs(sc - oct_.scale) <= 1e-12 * abs(oct_.scale), "%s: scale %r != %r" % (what, sc, oct_.scale)


def make_pair(name, seed, rotations=(), conj=True):
    import pytest
    K = pytest.importorskip("paper_2312_04356_gb300.ckks")
    P = oracle_params(name)
    o = Oracle(P, seed)
    o.gen_relin_key()
    if conj:
        o.gen_conj_key()
    o.gen_rotation_keys(rotations)
    ctx = gpu_ctx(name, seed)
    keys = K.ckks_keygen(ctx, list(rotations), conj)
    return K, o, ctx, keys
