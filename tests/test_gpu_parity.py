"""GPU parity: the CUDA library against the oracle, bit-exact on every limb.

Inputs are the seeded arrays of workloads.py; keys and encryption randomness come
from the same seed on both sides (each implements SplitMix64 itself).  Plaintexts
the oracle encodes are imported with *_import_rns so that both sides multiply by
identical integers (the FP64 encoders are compared separately, approximately).
"""
import math

import numpy as np
import pytest

import workloads as WL
from oracle import boot as BT
from oracle import encoding as E
from tests.pairs import assert_ct_equal, gpu_ctx, import_ct, import_plan, import_pt, make_pair, oracle_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()


@pytest.mark.parametrize("name", ["cfg1", "cfg2"])
def test_chain_matches_oracle(name):
    from paper_2312_04356_gb300 import ckks as K
    P = oracle_params(name)
    ctx = gpu_ctx(name, 1)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    assert q == list(P.q) and p == list(P.p)
    assert psi == list(P.psi_q) + list(P.psi_p)
    assert delta == list(P.delta)
    from oracle import _clib as C
    assert (K.ckks_ctx_gauss_table(ctx) == C.gauss_table(P.sigma)).all()


@pytest.mark.parametrize("name", ["cfg1", "cfg2"])
def test_ntt_bitexact(name):
    from oracle import _clib as C
    from paper_2312_04356_gb300 import ckks as K
    P = oracle_params(name)
    ctx = gpu_ctx(name, 1)
    ids = list(range(P.n_q)) + [P.n_q + j for j in range(P.n_p)]
    ids = ids[:6] + ids[-2:]
    mods = [(list(P.q) + list(P.p))[i] for i in ids]
    psis = [(list(P.psi_q) + list(P.psi_p))[i] for i in ids]
    x = WL.residues(3, mods, P.n)
    want = C.ntt_forward(x, mods, psis, P.logn)
    for variant in (-1, 0, 1, 2, 3, 4, 5):    # every launch variant the autotuner may pick
        K.ckks_ctx_set_ntt_variant(ctx, variant)
        dev = torch.from_numpy(x.view(np.int64).copy()).cuda()
        K.ckks_ntt_forward(ctx, dev.data_ptr(), len(ids), ids)
        torch.cuda.synchronize()
        got = dev.cpu().numpy().view(np.uint64)
        assert (got == want).all(), variant
        K.ckks_ntt_inverse(ctx, dev.data_ptr(), len(ids), ids)
        torch.cuda.synchronize()
        assert (dev.cpu().numpy().view(np.uint64) == x).all(), variant
    K.ckks_ctx_set_ntt_choices(ctx, [5, 4, 3, 2, 1, 0, 5, 4])   # one variant per size class
    dev = torch.from_numpy(x.view(np.int64).copy()).cuda()
    K.ckks_ntt_forward(ctx, dev.data_ptr(), len(ids), ids)
    torch.cuda.synchronize()
    assert (dev.cpu().numpy().view(np.uint64) == want).all()
    K.ckks_ctx_set_ntt_variant(ctx, -1)
    if P.logn == 16:
        choice = K.ckks_autotune(ctx, 1)
        assert all(c in (0, 1, 2, 3, 4, 5) for c in choice)
        K.ckks_ctx_set_ntt_choices(ctx, choice)
    # edge values: all zeros, all q-1
    e = np.stack([np.full(P.n, q - 1, dtype=np.uint64) for q in mods])
    e[0] = 0
    dev = torch.from_numpy(e.view(np.int64).copy()).cuda()
    K.ckks_ntt_forward(ctx, dev.data_ptr(), len(ids), ids)
    torch.cuda.synchronize()
    assert (dev.cpu().numpy().view(np.uint64) == C.ntt_forward(e, mods, psis, P.logn)).all()


def test_cluster_ntt_in_key_switching():
    """the one-launch cluster NTT forced for every size (1- and 3-limb transforms round-trip;
    the limb-list transforms of ModUp, ModDown and the key switch): hoisted rotations at
    N = 2^16 stay bit-exact against the oracle.  Then every two-pass variant forced in turn,
    and the default: hoisted rotations, HMult + relinearisation (ModDown) and rescale
    bit-exact at N = 2^16.  Every variant, the cluster one included: the level drop by
    rescales with integer factors (the inverse transform that reads the top limbs where they
    lie and applies the factor with N^-1) and ModRaise"""
    K, o, ctx, keys = make_pair("cfg2", 7, rotations=[1, 5], conj=False)
    P = o.P
    K.ckks_ctx_set_ntt_variant(ctx, 5)
    for nl in (1, 3):
        ids = list(range(nl))
        mods = [int(P.q[i]) for i in ids]
        x = WL.residues(11 + nl, mods, P.n)
        dev = torch.from_numpy(x.view(np.int64).copy()).cuda()
        K.ckks_ntt_forward(ctx, dev.data_ptr(), nl, ids)
        K.ckks_ntt_inverse(ctx, dev.data_ptr(), nl, ids)
        torch.cuda.synchronize()
        assert (dev.cpu().numpy().view(np.uint64) == x).all(), nl
    lev = 20
    z = WL.slots(12, P.n // 2, 0.3)
    ct = o.encrypt(o.encode_pt(z, lev, P.delta[lev]), 4)
    g = import_ct(K, ctx, ct)
    rots = K.ckks_rotate_hoisted(ctx, keys, g, [1, 5])
    want_rot = [o.rotate(ct, r) for r in (1, 5)]
    for r, gr, w in zip((1, 5), rots, want_rot):
        assert_ct_equal(K, ctx, gr, w, "rotation %d" % r)
    want_rs = o.rescale(ct)
    want_hm = o.mul_relin(ct, ct)
    for v in (0, 1, 2, 3, 4, -1):
        K.ckks_ctx_set_ntt_variant(ctx, v)
        for r, gr, w in zip((1, 5), K.ckks_rotate_hoisted(ctx, keys, g, [1, 5]), want_rot):
            assert_ct_equal(K, ctx, gr, w, "rotation %d, variant %d" % (r, v))
        assert_ct_equal(K, ctx, K.ckks_rescale(ctx, g), want_rs, "rescale, variant %d" % v)
        assert_ct_equal(K, ctx, K.ckks_mul_relin(ctx, keys, g, g), want_hm, "HMult, variant %d" % v)
    want_ld = o.level_down(ct, lev - 2)
    x0 = o.mod_drop(ct, 0)
    g0 = import_ct(K, ctx, x0)
    want_mr = o.mod_raise(x0)
    for v in (5, 0, 1, 2, 3, 4, -1):
        K.ckks_ctx_set_ntt_variant(ctx, v)
        assert_ct_equal(K, ctx, K.ckks_level_down(ctx, g, lev - 2), want_ld, "level drop, variant %d" % v)
        assert_ct_equal(K, ctx, K.ckks_mod_raise(ctx, g0), want_mr, "ModRaise, variant %d" % v)
    K.ckks_ctx_set_ntt_variant(ctx, -1)


def test_keys_encrypt_decrypt_bitexact():
    K, o, ctx, keys = make_pair("cfg1", 11, rotations=[1, 5])
    assert (K.ckks_keys_export_secret(ctx, keys) == o.s).all()
    P = o.P
    z = WL.slots(5, P.n // 2)
    for lev in (P.L, 1):
        pt = o.encode_pt(z, lev, P.delta[lev])
        gpt = import_pt(K, ctx, pt)
        assert (K.ckks_pt_export_rns(ctx, gpt) == pt.limbs).all()
        ct = o.encrypt(pt, 9)
        gct = K.ckks_encrypt(ctx, keys, gpt, 9)
        assert_ct_equal(K, ctx, gct, ct, "pk encryption")
        ct2 = o.encrypt_sk(pt, 10)
        gct2 = K.ckks_encrypt_sk(ctx, keys, gpt, 10)
        assert_ct_equal(K, ctx, gct2, ct2, "sk encryption")
        dec = K.ckks_decrypt(ctx, keys, gct)
        assert (K.ckks_pt_export_rns(ctx, dec) == o.decrypt(ct).limbs).all()
        # library decode of the decryption: back to the slots
        assert np.abs(K.ckks_decode(ctx, dec) - z).max() < 1e-6


def test_ops_bitexact():
    K, o, ctx, keys = make_pair("cfg1", 12, rotations=[1, 3, 100, 2047])
    P = o.P
    L = P.L
    z = WL.slots(6, P.n // 2, 0.5)
    ct = o.encrypt(o.encode_pt(z, L, P.delta[L]), 1)
    gct = import_ct(K, ctx, ct)
    assert_ct_equal(K, ctx, gct, ct, "import/export")
    assert_ct_equal(K, ctx, K.ckks_rescale(ctx, gct), o.rescale(ct), "rescale")
    assert_ct_equal(K, ctx, K.ckks_mul_relin(ctx, keys, gct, gct), o.mul_relin(ct, ct), "HMult")
    steps = [0, 1, 3, 100, 2047]
    gouts = K.ckks_rotate_hoisted(ctx, keys, gct, steps)
    for s, g, w in zip(steps, gouts, o.rotate_hoisted(ct, steps)):
        assert_ct_equal(K, ctx, g, w, "HRot %d" % s)
    assert_ct_equal(K, ctx, K.ckks_conjugate(ctx, keys, gct), o.conjugate(ct), "conj")
    assert_ct_equal(K, ctx, K.ckks_imult(ctx, gct), o.imult(ct), "imult")
    assert_ct_equal(K, ctx, K.ckks_mul_int(ctx, gct, -12345), o.mul_int(ct, -12345), "mul_int")
    assert_ct_equal(K, ctx, K.ckks_add_const(ctx, gct, 0.3), o.add_const(ct, 0.3), "add_const")
    assert_ct_equal(K, ctx, K.ckks_level_down(ctx, gct, 1), o.level_down(ct, 1), "level_down")
    c0 = o.mod_drop(ct, 0)
    assert_ct_equal(K, ctx, K.ckks_mod_raise(ctx, import_ct(K, ctx, c0)), o.mod_raise(c0), "ModRaise")
    pt = o.encode_pt(WL.slots(8, P.n // 2), L, float(P.q[L]))
    assert_ct_equal(K, ctx, K.ckks_mul_plain(ctx, gct, import_pt(K, ctx, pt)), o.mul_plain(ct, pt), "PMult")


def test_cfg1_conv_bitexact_and_fp64():
    """config 1: N=2^12, one 16x16 channel, 3x3 conv by the fused CinS BSGS; bit-exact limbs and
    decoded output vs FP64 conv2d within 2^-12"""
    P = oracle_params("cfg1")
    spec = WL.CONV["cfg1"]
    x = WL.image(1, spec["cin"], spec["w0"])
    W = WL.weights(1, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    w = E.pad_width(spec["w0"], spec["f"])
    C = P.n // (w * w)
    from oracle.scheme import Oracle
    o0 = Oracle(P, 21)
    plan = o0.conv_plan(W, 1, 1, 3, w, P.L, (P.delta[P.L - 1] * float(P.q[P.L])) / P.delta[P.L])
    K, o, ctx, keys = make_pair("cfg1", 21, rotations=plan.rotations(P.n // 2))
    pt = o.encode_pt(E.cins_input_slots(x, w, P.n), P.L, P.delta[P.L])
    ct = o.encrypt(pt, 4)
    gct = K.ckks_encrypt(ctx, keys, import_pt(K, ctx, pt), 4)
    out = o.conv2d_cins(ct, plan)
    gout = K.ckks_conv2d_cins(ctx, keys, gct, import_plan(K, ctx, plan))
    assert_ct_equal(K, ctx, gout, out, "fused conv")
    ref = E.conv2d_same(x, W)
    coeffs = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, gout), K.CKKS_COEFF)
    got = E.conv_output_from_coeffs(coeffs, C, w * w, 1, w, spec["w0"])
    assert np.abs(got - ref).max() < 2.0 ** -12
    # the library's own FP64 path: encoder and fused diagonals, decoded against FP64
    gps = K.ckks_ptset_conv_fused(ctx, W, 1, 1, 3, w, P.L, plan.scale)
    assert K.ckks_ptset_info(gps)["n_pts"] == len(plan.pts)
    gpt = K.ckks_encode(ctx, E.flatten_padded(x[0], w), P.L, P.delta[P.L], K.CKKS_CINS_REAL, w * w)
    own = K.ckks_conv2d_cins(ctx, keys, K.ckks_encrypt(ctx, keys, gpt, 5), gps)
    coeffs = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, own), K.CKKS_COEFF)
    got = E.conv_output_from_coeffs(coeffs, C, w * w, 1, w, spec["w0"])
    assert np.abs(got - ref).max() < 2.0 ** -12


def test_dwconv_bitexact_and_fp64():
    """depthwise conv: one PMult (Sec. 3.3.4) bit-exact against the oracle; the library's own
    kernel packing decodes to FP64 depthwise conv2d"""
    K, o, ctx, keys = make_pair("cfg2_small", 44, conj=False)
    P = o.P
    w0, w, f = 5, 8, 3
    C = P.n // (w * w)
    x = WL.image(44, C, w0)
    Kw = np.random.default_rng(44).normal(0, 0.3, (C, f, f))
    lev = 3
    pt = o.encode_pt(E.cins_input_slots(x, w, P.n), lev, P.delta[lev])
    pk = o.encode_pt(E.dwconv_kernel_slots(Kw, w, P.n), lev, P.delta[lev])
    ct = o.encrypt(pt, 1)
    want = o.dwconv_cins(ct, pk)
    got = K.ckks_dwconv_cins(ctx, import_ct(K, ctx, ct), import_pt(K, ctx, pk))
    assert_ct_equal(K, ctx, got, want, "dwconv")
    gk = K.ckks_encode_dwconv_kernel(ctx, Kw, w, lev, P.delta[lev])
    gx = K.ckks_encode_image(ctx, x, w, lev, P.delta[lev])
    own = K.ckks_dwconv_cins(ctx, K.ckks_encrypt(ctx, keys, gx, 2), gk)
    dec = K.ckks_decode_image(ctx, K.ckks_decrypt(ctx, keys, own), C, w0, w)
    assert np.abs(dec - E.dwconv_same(x, Kw)).max() < 2.0 ** -12


def test_own_encoder_close_to_oracle():
    """the library's FP64 encoder rounds to the same integers up to +-1"""
    K, o, ctx, keys = make_pair("cfg1", 3)
    P = o.P
    z = WL.slots(9, P.n // 2)
    g = K.ckks_pt_export_rns(ctx, K.ckks_encode(ctx, z, 2, P.delta[2]))
    w = o.encode_pt(z, 2, P.delta[2]).limbs
    for i in range(3):
        d = (g[i].astype(object) - w[i].astype(object)) % int(P.q[i])
        d = np.minimum(d, int(P.q[i]) - d)
        assert max(d) <= 1


def _block_pair(name, seed, import_all=True, oracle_all_keys=True, splits=None):
    P = oracle_params(name)
    spec = WL.CONV[name]
    x = WL.image(seed, spec["cin"], spec["w0"])
    W = WL.weights(seed, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    w = E.pad_width(spec["w0"], spec["f"])
    from oracle.scheme import Oracle
    o0 = Oracle(P, seed)
    ctos_B, stoc_B = splits if splits else (None, None)
    cfg = BT.BootConfig(o0, w, spec["w0"], spec["cout"], ctos_B=ctos_B, stoc_B=stoc_B)
    plan = o0.conv_plan(W, spec["cin"], spec["cout"], spec["f"], w, 1, (cfg.delta0 * float(P.q[1])) / P.delta[1])
    rots = BT.block_rotations(o0, plan, cfg)
    if oracle_all_keys:
        K, o, ctx, keys = make_pair(name, seed, rotations=rots)
    else:
        # the oracle only runs the conv here: it needs the conv's rotation keys alone
        from paper_2312_04356_gb300 import ckks as K
        o = Oracle(P, seed)
        o.gen_rotation_keys(plan.rotations(P.n // 2))
        ctx = gpu_ctx(name, seed)
        keys = K.ckks_keygen(ctx, rots, True)
    bt = K.ckks_boot_create(ctx, w, spec["w0"], spec["cout"])
    if splits:
        K.ckks_boot_set_bsgs_splits(ctx, bt, list(ctos_B) + list(stoc_B))
        assert K.ckks_boot_bsgs_splits(bt) == list(ctos_B) + list(stoc_B)
    info = K.ckks_boot_info(bt)
    assert info["c_drop"] == cfg.c_drop and info["K_eff"] == cfg.K_eff and info["s_raise"] == cfg.s_raise
    assert info["l_em"] == cfg.l_em and info["l_out"] == cfg.l_out and info["s_mask"] == cfg.s_mask
    assert sorted(K.ckks_boot_rotations(bt)) == sorted(set(r for p in cfg.ctos + cfg.stoc
                                                          for r in p.rotations(P.n // 2)))
    if import_all:
        for i, p in enumerate(cfg.ctos):
            K.ckks_boot_set_ctos(ctx, bt, i, import_plan(K, ctx, p))
        for i, p in enumerate(cfg.stoc):
            K.ckks_boot_set_stoc(ctx, bt, i, import_plan(K, ctx, p))
        K.ckks_boot_set_coeffs(ctx, bt, cfg.coeffs)
        K.ckks_boot_set_masks(ctx, bt, import_pt(K, ctx, cfg.pt_mask_re), import_pt(K, ctx, cfg.pt_mask_im))
    pt = o.encode_pt(E.cins_input_slots(x, w, P.n), 1, P.delta[1])
    return dict(K=K, o=o, ctx=ctx, keys=keys, cfg=cfg, plan=plan, bt=bt, pt=pt, x=x, W=W, w=w, spec=spec, P=P)


def _expected_slots(d):
    P, w, spec = d["P"], d["w"], d["spec"]
    conv = E.conv2d_same(d["x"], d["W"])
    return E.cins_input_slots(conv[: spec["cout"]], w, P.n), conv


def _pixels(d, slots):
    P, w = d["P"], d["w"]
    ell = w * w // 2
    C = P.n // (w * w)
    return np.stack([E.encode(slots[i * ell:(i + 1) * ell], w * w) for i in range(C)])


def test_block_small_bitexact():
    """the whole Alg. 1 block (conv -> ModRaise -> CtoS -> EvalMod x2 -> mask -> StoC1) on the
    config-2 chain at N = 2^10: bit-exact ciphertext and decoded error <= 2^-12, with
    dependent (default) and plain kernel launches, with and without side streams"""
    d = _block_pair("cfg2_small", 31)
    K, o, ctx, keys = d["K"], d["o"], d["ctx"], d["keys"]
    ct = o.encrypt(d["pt"], 2)
    gct = K.ckks_encrypt(ctx, keys, import_pt(K, ctx, d["pt"]), 2)
    gplan = import_plan(K, ctx, d["plan"])
    x0 = o.conv2d_cins(ct, d["plan"])
    gx0 = K.ckks_conv2d_cins(ctx, keys, gct, gplan)
    assert_ct_equal(K, ctx, gx0, x0, "conv")
    re, im = BT.bootstrap(o, x0, d["cfg"])
    gre, gim = K.ckks_bootstrap(ctx, keys, d["bt"], gx0)
    assert_ct_equal(K, ctx, gre, re, "EvalMod Re")
    assert_ct_equal(K, ctx, gim, im, "EvalMod Im")
    out = BT.stoc1(o, re, im, d["cfg"])
    gout = K.ckks_stoc1(ctx, keys, gre, gim, d["bt"])
    assert_ct_equal(K, ctx, gout, out, "StoC1")
    gblk = K.ckks_block(ctx, keys, gct, gplan, d["bt"])
    assert_ct_equal(K, ctx, gblk, out, "block")
    K.ckks_ctx_set_pdl(ctx, 0)                     # plain launches: the same residues
    gblk0 = K.ckks_block(ctx, keys, gct, gplan, d["bt"])
    K.ckks_ctx_set_pdl(ctx, 1)
    assert (K.ckks_ct_export_rns(ctx, gblk0) == K.ckks_ct_export_rns(ctx, gblk)).all()
    K.ckks_ctx_set_side_streams(ctx, 0)            # everything on one stream: the same residues
    gblk1 = K.ckks_block(ctx, keys, gct, gplan, d["bt"])
    K.ckks_ctx_set_side_streams(ctx, 1)
    assert (K.ckks_ct_export_rns(ctx, gblk1) == K.ckks_ct_export_rns(ctx, gblk)).all()
    K.ckks_ctx_set_inner_batching(ctx, 1)          # Chebyshev generations as lockstep batches
    gblk2 = K.ckks_block(ctx, keys, gct, gplan, d["bt"])
    K.ckks_ctx_set_inner_batching(ctx, 0)
    assert (K.ckks_ct_export_rns(ctx, gblk2) == K.ckks_ct_export_rns(ctx, gblk)).all()
    zexp, _ = _expected_slots(d)
    got = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, gblk))
    assert np.abs(_pixels(d, got) - _pixels(d, zexp)).max() < 2.0 ** -12


def test_block_bsgs_splits_bitexact():
    """every CtoS / StoC1 level evaluated with B = 2 and B = 4 baby steps instead of the
    cost-model choice: the rotation set follows the splits and the block stays bit-exact
    against the oracle built with the same splits"""
    for B in (2, 4):
        d = _block_pair("cfg2_small", 34, splits=([B] * 3, [B] * 3))
        K, o, ctx, keys = d["K"], d["o"], d["ctx"], d["keys"]
        assert [p.B for p in d["cfg"].ctos + d["cfg"].stoc] == [B] * 6
        ct = o.encrypt(d["pt"], 2)
        gct = K.ckks_encrypt(ctx, keys, import_pt(K, ctx, d["pt"]), 2)
        out = BT.block(o, ct, d["plan"], d["cfg"])
        gblk = K.ckks_block(ctx, keys, gct, import_plan(K, ctx, d["plan"]), d["bt"])
        assert_ct_equal(K, ctx, gblk, out, "block with B = %d" % B)


def test_bsgs_split_autotuner():
    """the autotuner picks one baby-step count per level among the timed candidates, leaves
    the op counters alone, and the tuned block (the library's own plans and keys for the
    tuned rotation set) decodes within 2^-12; the rotation set is the oracle's for the
    same splits"""
    from paper_2312_04356_gb300 import ckks as K
    from oracle.scheme import Oracle, boot_bsgs_B
    P = oracle_params("cfg2_small")
    spec = WL.CONV["cfg2_small"]
    w = E.pad_width(spec["w0"], spec["f"])
    ctx = gpu_ctx("cfg2_small", 35)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    bt = K.ckks_boot_create(ctx, w, spec["w0"], spec["cout"])
    before = K.ckks_ctx_counters(ctx)
    B = K.ckks_boot_tune_bsgs(ctx, bt, 2)
    assert K.ckks_ctx_counters(ctx) == before
    cfg = BT.BootConfig(Oracle(P, 35), w, spec["w0"], spec["cout"], ctos_B=B[:3], stoc_B=B[3:])
    for b, pl in zip(B, cfg.ctos + cfg.stoc):
        assert b in [c for c in (2, 4, 8, 16, 32) if c <= min(pl.count, 32)] + [boot_bsgs_B(pl.count)]
    assert K.ckks_boot_bsgs_splits(bt) == B
    assert sorted(K.ckks_boot_rotations(bt)) == sorted(set(r for pl in cfg.ctos + cfg.stoc
                                                           for r in pl.rotations(P.n // 2)))
    W = WL.weights(35, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    x = WL.image(35, spec["cin"], spec["w0"])
    conv = K.ckks_ptset_conv_fused(ctx, W, spec["cin"], spec["cout"], spec["f"], w, 1, (cfg.delta0 * q[1]) / delta[1])
    keys = K.ckks_keygen(ctx, sorted(set(K.ckks_ptset_rotations(conv)) | set(K.ckks_boot_rotations(bt))), True)
    ct = K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, x, w, 1, delta[1]), 3)
    out = K.ckks_block(ctx, keys, ct, conv, bt)
    got = K.ckks_decode_image(ctx, K.ckks_decrypt(ctx, keys, out), spec["cout"], spec["w0"], w)
    assert np.abs(got - E.conv2d_same(x, W)[: spec["cout"]]).max() < 2.0 ** -12


def test_block_graph_replays_bitexact():
    """the block recorded as a CUDA graph gives the eager block's ciphertext on every replay,
    also for a new input written into the same handle"""
    d = _block_pair("cfg2_small", 33)
    K, o, ctx0, keys0 = d["K"], d["o"], d["ctx"], d["keys"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = gpu_ctx("cfg2_small", 33)
        keys = K.ckks_keygen(ctx, K.ckks_boot_rotations(d["bt"]) + [d["w"] ** 2 // 2 * k for k in range(1, 16)], True)
        bt = K.ckks_boot_create(ctx, d["w"], d["spec"]["w0"], d["spec"]["cout"])
        spec = d["spec"]
        conv = K.ckks_ptset_conv_fused(ctx, d["W"], spec["cin"], spec["cout"], spec["f"], d["w"], 1, d["plan"].scale)
        ct = K.ckks_encrypt(ctx, keys, import_pt(K, ctx, d["pt"]), 2)
        want = K.ckks_ct_export_rns(ctx, K.ckks_block(ctx, keys, ct, conv, bt))
        out = K.ckks_ct_create(ctx)
        g = K.ckks_block_graph_create(ctx, keys, ct, conv, bt, out)
        assert K.ckks_graph_info(g) > 100
        for _ in range(2):
            K.ckks_graph_launch(g)
            K.ckks_sync(ctx)
            assert (K.ckks_ct_export_rns(ctx, out) == want).all()
        K.ckks_ct_copy_into(ctx, K.ckks_encrypt(ctx, keys, import_pt(K, ctx, d["pt"]), 9), ct)   # new input
        want2 = K.ckks_ct_export_rns(ctx, K.ckks_block(ctx, keys, ct, conv, bt))
        K.ckks_graph_launch(g)
        K.ckks_sync(ctx)
        assert (K.ckks_ct_export_rns(ctx, out) == want2).all()


def test_block_small_own_plans():
    """same block with the library's own FP64 plans, masks and Chebyshev fit: decoded within 2^-12"""
    d = _block_pair("cfg2_small", 32, import_all=False)
    K, ctx, keys = d["K"], d["ctx"], d["keys"]
    gct = K.ckks_encrypt(ctx, keys, import_pt(K, ctx, d["pt"]), 2)
    spec = d["spec"]
    gplan = K.ckks_ptset_conv_fused(ctx, d["W"], spec["cin"], spec["cout"], spec["f"], d["w"], 1, d["plan"].scale)
    gblk = K.ckks_block(ctx, keys, gct, gplan, d["bt"])
    zexp, _ = _expected_slots(d)
    got = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, gblk))
    assert np.abs(_pixels(d, got) - _pixels(d, zexp)).max() < 2.0 ** -12


def test_eval_poly_bitexact():
    K, o, ctx, keys = make_pair("cfg2_small", 41)
    P = o.P
    y = np.random.default_rng(4).uniform(-1, 1, P.n // 2)
    pt = o.encode_pt(y, P.L, P.delta[P.L])
    ct = o.encrypt(pt, 1)
    coeffs = list(np.polynomial.chebyshev.chebinterpolate(lambda t: t * (1 + np.tanh(4 * t)) / 2, 15))
    coeffs = [c if k % 2 == 1 or k == 0 else 0.0 for k, c in enumerate(coeffs)]
    want = o.cheb_eval(ct, coeffs)
    got = K.ckks_eval_poly(ctx, keys, import_ct(K, ctx, ct), coeffs)
    assert_ct_equal(K, ctx, got, want, "eval_poly")


def test_eval_relu_bitexact():
    """HActivation: the (15, 15, 27) composite ReLU fitted by the oracle, bit-exact on the GPU,
    decoded within 2^-12 of the FP64 polynomial ReLU"""
    from oracle import relu as R
    stages, _ = R.composite_relu_stages()
    K, o, ctx, keys = make_pair("cfg2_small", 43)
    P = o.P
    v = np.random.default_rng(5).uniform(-1, 1, P.n // 2)
    ct = o.encrypt(o.encode_pt(v, P.L, P.delta[P.L]), 1)
    want = R.relu_eval(o, ct, stages)
    got = K.ckks_eval_relu(ctx, keys, import_ct(K, ctx, ct), stages)
    assert_ct_equal(K, ctx, got, want, "composite ReLU")
    dec = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, got)).real
    assert np.abs(dec - R.relu_poly_fp64(v, stages)).max() < 2.0 ** -12


def test_eval_relu_full_size_across_the_segment_boundary():
    """HActivation at N = 2^16 (config-2 chain) from the top level: the (15, 15, 27) composite
    crosses from the 48-bit bootstrapping segment into the 42-bit circuit segment, uses 18
    levels (one more than the stages' depth, as the header states) and decodes within 2^-12 of
    the FP64 polynomial ReLU"""
    from oracle import relu as R
    from paper_2312_04356_gb300 import ckks as K
    stages, _ = R.composite_relu_stages()
    P = oracle_params("cfg2")
    ctx = gpu_ctx("cfg2", 47)
    keys = K.ckks_keygen(ctx, [], False)
    v = np.random.default_rng(6).uniform(-1, 1, P.n // 2)
    ct = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, v, P.L, P.delta[P.L]), 3)
    got = K.ckks_eval_relu(ctx, keys, ct, stages)
    assert K.ckks_ct_info(got)[0] == P.L - 18
    dec = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, got)).real
    assert np.abs(dec - R.relu_poly_fp64(v, stages)).max() < 2.0 ** -12


@pytest.mark.slow
def test_cfg2_block_full_size():
    """config 2 at full size (N = 2^16, 24 limbs, 16 channels of 32x32, Gaussian weights):
    the conv output and the CtoS input are bit-exact against the oracle; the whole block
    decodes to the masked FP64 conv2d within 2^-12"""
    d = _block_pair("cfg2", 7, import_all=False, oracle_all_keys=False)
    K, o, ctx, keys = d["K"], d["o"], d["ctx"], d["keys"]
    ct = o.encrypt(d["pt"], 2)
    gct = K.ckks_encrypt(ctx, keys, import_pt(K, ctx, d["pt"]), 2)
    assert_ct_equal(K, ctx, gct, ct, "encryption")
    gplan = import_plan(K, ctx, d["plan"])
    x0 = o.conv2d_cins(ct, d["plan"])
    gx0 = K.ckks_conv2d_cins(ctx, keys, gct, gplan)
    assert_ct_equal(K, ctx, gx0, x0, "conv")
    assert_ct_equal(K, ctx, K.ckks_mod_raise(ctx, gx0), o.mod_raise(x0), "ModRaise")
    gblk = K.ckks_block(ctx, keys, gct, gplan, d["bt"])
    zexp, conv = _expected_slots(d)
    got = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, gblk))
    err = np.abs(_pixels(d, got) - _pixels(d, zexp)).max()
    assert err < 2.0 ** -12, err


@pytest.mark.slow
def test_cfg2_block_full_size_bitexact():
    """config 2 at full size (N = 2^16, 24 limbs, dnum 3, 16 channels of 32 x 32) with the BSGS
    splits the tuner picks on GB300 (CtoS 16 / 16 / 32, StoC1 16 / 16 / 8: the fused baby-step
    kernel with 4 and with 2 giant steps): every limb of the encryption, the fused conv, the
    bootstrap's EvalMod outputs (Re and Im: ModRaise, three CtoS HMatmuls, the conjugate split,
    the scale drop, the degree-59 Chebyshev series and three double angles, across the
    segment boundary), StoC1, the block as called (which skips the Im branch its zero mask
    removes) and the block replayed as the CUDA graph the bench times, against the oracle's
    block; decoded within 2^-12 of the masked FP64 conv2d"""
    s = torch.cuda.Stream()          # the graph needs a context on a non-default stream
    with torch.cuda.stream(s):
        _full_size_block(s)


def _full_size_block(s):
    d = _block_pair("cfg2", 7, splits=([16, 16, 32], [16, 16, 8]))
    K, o, ctx, keys = d["K"], d["o"], d["ctx"], d["keys"]
    ct = o.encrypt(d["pt"], 2)
    gct = K.ckks_encrypt(ctx, keys, import_pt(K, ctx, d["pt"]), 2)
    assert_ct_equal(K, ctx, gct, ct, "encryption")
    gplan = import_plan(K, ctx, d["plan"])
    x0 = o.conv2d_cins(ct, d["plan"])
    gx0 = K.ckks_conv2d_cins(ctx, keys, gct, gplan)
    assert_ct_equal(K, ctx, gx0, x0, "conv")
    re, im = BT.bootstrap(o, x0, d["cfg"])
    gre, gim = K.ckks_bootstrap(ctx, keys, d["bt"], gx0)
    assert_ct_equal(K, ctx, gre, re, "EvalMod Re")
    assert_ct_equal(K, ctx, gim, im, "EvalMod Im")
    out = BT.stoc1(o, re, im, d["cfg"])
    assert_ct_equal(K, ctx, K.ckks_stoc1(ctx, keys, gre, gim, d["bt"]), out, "StoC1")
    assert_ct_equal(K, ctx, K.ckks_block(ctx, keys, gct, gplan, d["bt"]), out, "block")
    gout = K.ckks_ct_create(ctx)
    g = K.ckks_block_graph_create(ctx, keys, gct, gplan, d["bt"], gout)
    K.ckks_graph_launch(g)
    K.ckks_sync(ctx)
    assert_ct_equal(K, ctx, gout, out, "block graph replay")
    zexp, _ = _expected_slots(d)
    got = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, gout))
    err = np.abs(_pixels(d, got) - _pixels(d, zexp)).max()
    assert err < 2.0 ** -12, err


# ------------------------------------------------- downsampling conv (Alg. 2) ----
def _ds_tail_slots(P, cfg, x, seed):
    """Re / Im slot vectors as the bootstrap hands them to the tail (slot i l + u: pixel
    rev_l(u), resp. rev_l(u) + l, of channel i, divided by the mask value); pixels outside the
    image carry noise that the masks remove"""
    g = np.random.default_rng(seed)
    val = float(P.q[0]) / (2.0 * np.pi * cfg.delta0)
    ell, w = cfg.ell, cfg.w
    rev = E.bitrev_indices(ell)
    re, im = np.zeros(P.n // 2), np.zeros(P.n // 2)
    for i in range(cfg.C):
        img = g.uniform(-1, 1, (w, w))
        if i < x.shape[0]:
            img[:cfg.w0, :cfg.w0] = x[i]
        f = img.reshape(-1)
        re[i * ell:(i + 1) * ell] = f[rev] / val
        im[i * ell:(i + 1) * ell] = f[rev + ell] / val
    return re, im


def _import_boot(K, ctx, bt, cfg):
    for i, p in enumerate(cfg.ctos):
        K.ckks_boot_set_ctos(ctx, bt, i, import_plan(K, ctx, p))
    for i, p in enumerate(cfg.stoc):
        K.ckks_boot_set_stoc(ctx, bt, i, import_plan(K, ctx, p))
    if cfg.decomp is not None:
        K.ckks_boot_set_decomp(ctx, bt, import_plan(K, ctx, cfg.decomp))
    K.ckks_boot_set_coeffs(ctx, bt, cfg.coeffs)
    K.ckks_boot_set_masks(ctx, bt, import_pt(K, ctx, cfg.pt_mask_re), import_pt(K, ctx, cfg.pt_mask_im))


def _ds_case(seed):
    """config-2 chain at N = 2^10: two ciphertexts of C = 16 channels (4 x 4 in w = 8) ->
    stride-2 conv -> 64 channels of 2 x 2 in w = 4"""
    P = oracle_params("cfg2_small")
    w0, w, f = 4, 8, 3
    C = P.n // (w * w)
    x = WL.image(seed, 2 * C, w0)
    W = WL.weights(seed, 4 * C, 2 * C, f, "normal")
    return P, w0, w, f, C, x, W


def test_downsample_bitexact():
    """Alg. 2 on both sides with the oracle's plaintexts: stride-2 tail (mask, Re + i Im,
    decomposition, S_{l/4<-1}) per input ciphertext, then the two decomposed convs + one
    bootstrap + tail: bit-exact ciphertexts, decoded output within 2^-12 of the FP64 stride-2
    conv2d"""
    from oracle.scheme import Oracle
    seed = 61
    P, w0, w, f, C, x, W = _ds_case(seed)
    o0 = Oracle(P, seed)
    cfg_in = BT.BootConfig(o0, w, w0, C, stride=2)
    cfg_out = BT.BootConfig(o0, w // 2, w0 // 2, 4 * C)
    m = P.n // 2
    conv_rots = {(d * (w * w // 8)) % m for d in range(1, 4 * C)}
    rots = sorted(set(BT.block_rotations(o0, None, cfg_in)) | set(BT.block_rotations(o0, None, cfg_out)) | conv_rots)
    K, o, ctx, keys = make_pair("cfg2_small", seed, rotations=rots)
    cfg_in = BT.BootConfig(o, w, w0, C, stride=2)
    cfg_out = BT.BootConfig(o, w // 2, w0 // 2, 4 * C)
    bt_in = K.ckks_boot_create(ctx, w, w0, C, stride=2)
    bt_out = K.ckks_boot_create(ctx, w // 2, w0 // 2, 4 * C)
    assert K.ckks_boot_info(bt_in)["l_out"] == cfg_in.l_out
    assert sorted(K.ckks_boot_rotations(bt_in)) == sorted(BT.block_rotations(o, None, cfg_in))
    _import_boot(K, ctx, bt_in, cfg_in)
    _import_boot(K, ctx, bt_out, cfg_out)
    ins, gins, gres, gims = [], [], [], []
    for t in range(2):
        re, im = _ds_tail_slots(P, cfg_in, x[t * C:(t + 1) * C], seed + t)
        cre = o.encrypt(o.encode_pt(re, cfg_in.l_em, cfg_in.s_em), 2 * t + 1)
        cim = o.encrypt(o.encode_pt(im, cfg_in.l_em, cfg_in.s_em), 2 * t + 2)
        y = BT.stoc1(o, cre, cim, cfg_in)
        gres.append(import_ct(K, ctx, cre))
        gims.append(import_ct(K, ctx, cim))
        gy = K.ckks_stoc1(ctx, keys, gres[-1], gims[-1], bt_in)
        assert_ct_equal(K, ctx, gy, y, "stride-2 tail %d" % t)
        ins.append(o.level_down(y, 1))
        gins.append(K.ckks_level_down(ctx, gy, 1))
        assert_ct_equal(K, ctx, gins[-1], ins[-1], "level_down %d" % t)
    s_pt = (cfg_out.delta0 * float(P.q[1])) / ins[0].scale
    plans, gplans = [], []
    for t in range(2):
        Wt = E.decompose_kernels(W, C, t)
        plans.append(o.conv_plan(Wt, 4 * C, 4 * C, Wt.shape[2], w // 2, 1, s_pt))
        gplans.append(import_plan(K, ctx, plans[-1]))
    out = BT.block_multi(o, ins, plans, cfg_out)
    gout = K.ckks_block_multi(ctx, keys, gins, gplans, bt_out)
    assert_ct_equal(K, ctx, gout, out, "Alg. 2 conv + bootstrap")
    assert_ct_equal(K, ctx, K.ckks_downsample_layer(ctx, keys, gres, gims, bt_in, gplans, bt_out), out,
                    "Alg. 2 layer")
    got = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, gout))
    ref = E.conv2d_stride2(x, W)
    w2 = w // 2
    ell2 = w2 * w2 // 2
    pix = np.stack([E.encode(got[i * ell2:(i + 1) * ell2], w2 * w2) for i in range(4 * C)])
    want = np.stack([E.flatten_padded(v, w2) for v in ref])
    assert np.abs(pix - want).max() < 2.0 ** -12


def test_downsample_own_plans():
    """the library's own decomposition, S_{l/4<-1}, masks, EvalMod fit and decomposed conv sets
    (ckks_ptset_conv_fused_s2) with its own encoder: decoded within 2^-12 of the FP64 stride-2
    conv; the layer recorded as a CUDA graph replays the eager layer's ciphertext"""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _downsample_own_plans()


def _downsample_own_plans():
    from oracle.scheme import Oracle
    from paper_2312_04356_gb300 import ckks as K
    seed = 62
    P, w0, w, f, C, x, W = _ds_case(seed)
    ctx = gpu_ctx("cfg2_small", seed)
    m = P.n // 2
    bt_in = K.ckks_boot_create(ctx, w, w0, C, stride=2)
    bt_out = K.ckks_boot_create(ctx, w // 2, w0 // 2, 4 * C)
    conv_rots = {(d * (w * w // 8)) % m for d in range(1, 4 * C)}
    keys = K.ckks_keygen(ctx, sorted(set(K.ckks_boot_rotations(bt_in)) | set(K.ckks_boot_rotations(bt_out))
                                     | conv_rots), True)
    info = K.ckks_boot_info(bt_in)
    o0 = Oracle(P, seed)
    cfg_in = BT.BootConfig(o0, w, w0, C, stride=2)      # layout only: s_em, l_em, mask value
    assert info["l_em"] == cfg_in.l_em and info["s_em"] == cfg_in.s_em
    gins, gres, gims = [], [], []
    for t in range(2):
        re, im = _ds_tail_slots(P, cfg_in, x[t * C:(t + 1) * C], seed + t)
        gres.append(K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, re, cfg_in.l_em, cfg_in.s_em), 2 * t + 1))
        gims.append(K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, im, cfg_in.l_em, cfg_in.s_em), 2 * t + 2))
        gins.append(K.ckks_level_down(ctx, K.ckks_stoc1(ctx, keys, gres[-1], gims[-1], bt_in), 1))
    lev, sc = K.ckks_ct_info(gins[0])
    s_pt = (2.0 ** 49 * float(P.q[1])) / sc
    gplans = [K.ckks_ptset_conv_fused_s2(ctx, W, 2 * C, 4 * C, f, w, t, 1, s_pt) for t in range(2)]
    gout = K.ckks_block_multi(ctx, keys, gins, gplans, bt_out)
    want = K.ckks_ct_export_rns(ctx, gout)
    assert (K.ckks_ct_export_rns(ctx, K.ckks_downsample_layer(ctx, keys, gres, gims, bt_in, gplans, bt_out))
            == want).all()
    gout2 = K.ckks_ct_create(ctx)
    g = K.ckks_downsample_layer_graph_create(ctx, keys, gres, gims, bt_in, gplans, bt_out, gout2)
    for _ in range(2):
        K.ckks_graph_launch(g)
        K.ckks_sync(ctx)
        assert (K.ckks_ct_export_rns(ctx, gout2) == want).all()
    got = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, gout))
    ref = E.conv2d_stride2(x, W)
    w2 = w // 2
    ell2 = w2 * w2 // 2
    pix = np.stack([E.encode(got[i * ell2:(i + 1) * ell2], w2 * w2) for i in range(4 * C)])
    want = np.stack([E.flatten_padded(v, w2) for v in ref])
    assert np.abs(pix - want).max() < 2.0 ** -12


def test_downsample_dwconv_and_avgpool():
    """downsampling depthwise conv and stride-2 average pooling (Sec. 3.3.4) through Alg. 2:
    the library's depthwise sets (ckks_ptset_dwconv_fused_s2) give the same ciphertext as the
    general stride-2 sets with the diagonal weights, and decode within 2^-12 of the FP64
    strided depthwise conv / average pooling; channels without a kernel decode to zero"""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _downsample_dwconv_avgpool()


def _downsample_dwconv_avgpool():
    from oracle.scheme import Oracle
    from paper_2312_04356_gb300 import ckks as K
    seed = 63
    P, w0, w, f, C, x, _ = _ds_case(seed)
    ctx = gpu_ctx("cfg2_small", seed)
    m = P.n // 2
    bt_in = K.ckks_boot_create(ctx, w, w0, C, stride=2)
    bt_out = K.ckks_boot_create(ctx, w // 2, w0 // 2, 4 * C)
    conv_rots = {(d * (w * w // 8)) % m for d in range(1, 4 * C)}
    keys = K.ckks_keygen(ctx, sorted(set(K.ckks_boot_rotations(bt_in)) | set(K.ckks_boot_rotations(bt_out))
                                     | conv_rots), True)
    cfg_in = BT.BootConfig(Oracle(P, seed), w, w0, C, stride=2)      # layout only
    gins = []
    for t in range(2):
        re, im = _ds_tail_slots(P, cfg_in, x[t * C:(t + 1) * C], seed + t)
        gre = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, re, cfg_in.l_em, cfg_in.s_em), 2 * t + 1)
        gim = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, im, cfg_in.l_em, cfg_in.s_em), 2 * t + 2)
        gins.append(K.ckks_level_down(ctx, K.ckks_stoc1(ctx, keys, gre, gim, bt_in), 1))
    lev, sc = K.ckks_ct_info(gins[0])
    s_pt = (2.0 ** 49 * float(P.q[1])) / sc
    c = 2 * C
    Kd = np.random.default_rng(seed).normal(0.0, 0.3, (c, f, f))
    Ka = np.full((c, f, f), 1.0 / (f * f))
    w2 = w // 2
    ell2 = w2 * w2 // 2

    def run(plans):
        return K.ckks_block_multi(ctx, keys, gins, plans, bt_out)

    def decoded_pixels(ct):
        got = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, ct))
        return np.stack([E.encode(got[i * ell2:(i + 1) * ell2], w2 * w2) for i in range(4 * C)])

    def diag_weights(k):
        Wd = np.zeros((c, c, f, f))
        Wd[np.arange(c), np.arange(c)] = k
        return Wd

    gdw = run([K.ckks_ptset_dwconv_fused_s2(ctx, Kd, w, t, 1, s_pt) for t in range(2)])
    gfull = run([K.ckks_ptset_conv_fused_s2(ctx, diag_weights(Kd), c, c, f, w, t, 1, s_pt) for t in range(2)])
    assert (K.ckks_ct_export_rns(ctx, gdw) == K.ckks_ct_export_rns(ctx, gfull)).all()
    for ct, k in ((gdw, Kd), (run([K.ckks_ptset_dwconv_fused_s2(ctx, Ka, w, t, 1, s_pt) for t in range(2)]), Ka)):
        pix = decoded_pixels(ct)
        want = np.stack([E.flatten_padded(v, w2) for v in E.conv2d_stride2(x, diag_weights(k))])
        assert np.abs(pix[:c] - want).max() < 2.0 ** -12
        assert np.abs(pix[c:]).max() < 2.0 ** -12


def test_fc_stoc_bitexact_and_fp64():
    """FC fused with the whole StoC (Sec. 4.3): replication rotations + BSGS over the n_in
    diagonals of V M, bit-exact against the oracle; the library's own set decodes (coefficient
    encoding) to M x"""
    from oracle.scheme import Oracle
    seed = 81
    P = oracle_params("cfg2_small")
    m = P.n // 2
    n_in, n_out = 16, 40
    M = np.random.default_rng(seed).normal(0, 0.3, (n_out, n_in))
    x = np.zeros(m)
    x[:n_in] = WL.slots(seed, n_in).real
    lev = 3
    o0 = Oracle(P, seed)
    plan = o0.fc_plan(M, lev, (P.delta[lev - 1] * float(P.q[lev])) / P.delta[lev])
    K, o, ctx, keys = make_pair("cfg2_small", seed, rotations=plan.rotations(m) + o0.fc_replicate_steps(n_in),
                                conj=False)
    pt = o.encode_pt(x, lev, P.delta[lev])
    ct = o.encrypt(pt, 3)
    want = o.fc_stoc(ct, plan, n_in)
    got = K.ckks_fc_stoc(ctx, keys, import_ct(K, ctx, ct), import_plan(K, ctx, plan), n_in)
    assert_ct_equal(K, ctx, got, want, "FC (x) StoC")
    own = K.ckks_ptset_fc_stoc(ctx, M, lev, plan.scale)
    gct = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, x, lev, P.delta[lev]), 4)
    y = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, K.ckks_fc_stoc(ctx, keys, gct, own, n_in)), K.CKKS_COEFF)
    assert np.abs(y[:n_out] - M @ x[:n_in]).max() < 2.0 ** -12
    assert np.abs(y[n_out:]).max() < 2.0 ** -12


def test_eval_poly_interval_and_power_basis():
    """ckks_eval_poly on [0, 4] in the Chebyshev basis of the interval: bit-exact against the
    oracle (the change of variable y = (2x - a - b) / (b - a) costs one level); in the power
    basis on [-3, 1]: decoded against numpy's polynomial (the FP64 re-expression in the
    Chebyshev basis differs in its last bits between the two sides)"""
    K, o, ctx, keys = make_pair("cfg2_small", 45)
    P = o.P
    rng = np.random.default_rng(45)
    c = list(rng.normal(0, 0.3, 8))
    x = rng.uniform(0.0, 4.0, P.n // 2)
    ct = o.encrypt(o.encode_pt(x, P.L, P.delta[P.L]), 2)
    want = o.eval_poly(ct, c, 0.0, 4.0, "cheb")
    got = K.ckks_eval_poly(ctx, keys, import_ct(K, ctx, ct), c, K.CKKS_BASIS_CHEB, 0.0, 4.0)
    assert_ct_equal(K, ctx, got, want, "eval_poly on [0, 4]")
    x2 = rng.uniform(-3.0, 1.0, P.n // 2)
    ct2 = import_ct(K, ctx, o.encrypt(o.encode_pt(x2, P.L, P.delta[P.L]), 3))
    out = K.ckks_eval_poly(ctx, keys, ct2, c, K.CKKS_BASIS_POWER, -3.0, 1.0)
    dec = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, out)).real
    ref = np.polynomial.polynomial.polyval(x2, c)
    assert np.abs(dec - ref).max() < 1e-6 * max(1.0, np.abs(ref).max())
    with pytest.raises(K.CkksError):
        K.ckks_eval_poly(ctx, keys, ct2, c, K.CKKS_BASIS_POWER, 1.0, -3.0)      # a >= b
