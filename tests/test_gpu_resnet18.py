"""ImageNet-shaped (ResNet-18) layers on the GPU at N = 2^10 on the config-2 chain: the 7x7
stride-2 stem from client-encoded polyphase images (one input channel per ciphertext) and a
stage layer whose channels span several ciphertexts on both sides (Sec. 3.3.3).  Bit-exact
against the oracle with its plaintexts imported; with the library's own conv sets and
bootstrapping plans, decoded within 2^-12 of FP64 conv2d."""
import numpy as np
import pytest

from oracle import boot as BT
from oracle import encoding as E
from tests.pairs import assert_ct_equal, import_plan, import_pt, make_pair, oracle_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rng = np.random.default_rng(19)


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()


def _import_boot(K, ctx, bt, cfg):
    for i, p in enumerate(cfg.ctos):
        K.ckks_boot_set_ctos(ctx, bt, i, import_plan(K, ctx, p))
    for i, p in enumerate(cfg.stoc):
        K.ckks_boot_set_stoc(ctx, bt, i, import_plan(K, ctx, p))
    K.ckks_boot_set_coeffs(ctx, bt, cfg.coeffs)
    K.ckks_boot_set_masks(ctx, bt, import_pt(K, ctx, cfg.pt_mask_re), import_pt(K, ctx, cfg.pt_mask_im))


def _slots_pixels(K, ctx, keys, ct, w, cout):
    ell = w * w // 2
    z = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, ct))
    return np.stack([E.encode(z[i * ell:(i + 1) * ell], w * w) for i in range(cout)])


def test_stem_bitexact_and_own_sets():
    from oracle.scheme import Oracle
    P = oracle_params("cfg2_small")
    x = rng.random((3, 28, 28))
    W = rng.normal(0, 0.1, (4, 3, 7, 7))
    pp = E.decompose_images(x)
    w = 16
    o0 = Oracle(P, 61)
    cfg = BT.BootConfig(o0, w, 14, 4)
    s_pt = (cfg.delta0 * float(P.q[1])) / P.delta[1]
    plans = [o0.conv_plan(E.decompose_kernels(W, 1, t), 4, 4, 5, w, 1, s_pt) for t in range(3)]
    m = P.n // 2
    rots = sorted(set().union(*[set(p.rotations(m)) for p in plans]) | set(BT.block_rotations(o0, None, cfg)))
    K, o, ctx, keys = make_pair("cfg2_small", 61, rotations=rots)
    cfg = BT.BootConfig(o, w, 14, 4)
    pts = [o.encode_pt(E.cins_input_slots(pp[4 * t:4 * (t + 1)], w, P.n), 1, P.delta[1]) for t in range(3)]
    cts = [o.encrypt(pt, 5 + t) for t, pt in enumerate(pts)]
    want = BT.block_multi(o, cts, plans, cfg)
    gcts = [K.ckks_encrypt(ctx, keys, import_pt(K, ctx, pt), 5 + t) for t, pt in enumerate(pts)]
    bt = K.ckks_boot_create(ctx, w, 14, 4)
    _import_boot(K, ctx, bt, cfg)
    got = K.ckks_block_multi(ctx, keys, gcts, [import_plan(K, ctx, p) for p in plans], bt)
    assert_ct_equal(K, ctx, got, want, "stem block")
    # the library's own stride-2 sets (input width 32: one channel per ciphertext), encoder and plans
    bt2 = K.ckks_boot_create(ctx, w, 14, 4)
    own = [K.ckks_ptset_conv_fused_s2(ctx, W, 3, 4, 7, 2 * w, t, 1, s_pt) for t in range(3)]
    for ps in own:
        K.ckks_keys_add_rotations(ctx, keys, K.ckks_ptset_rotations(ps))
    K.ckks_keys_add_rotations(ctx, keys, K.ckks_boot_rotations(bt2))
    ins = [K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, pp[4 * t:4 * (t + 1)], w, 1, P.delta[1]), 9 + t)
           for t in range(3)]
    out = K.ckks_block_multi(ctx, keys, ins, own, bt2)
    ref = np.stack([E.flatten_padded(v, w) for v in E.conv2d_stride2(x, W)])
    assert np.abs(_slots_pixels(K, ctx, keys, out, w, 4) - ref).max() < 2.0 ** -12


def test_stage_layer_spanning_ciphertexts():
    """32 -> 32 channels of 4 x 4 (w = 8, C = 16: two ciphertexts in, two out): the first output
    ciphertext bit-exact against the oracle; every output with the library's own sets decoded
    within 2^-12 of FP64 conv2d"""
    from oracle.scheme import Oracle
    P = oracle_params("cfg2_small")
    w0, w, C = 4, 8, 16
    x = rng.random((2 * C, w0, w0))
    W = rng.normal(0, 0.1, (2 * C, 2 * C, 3, 3))
    o0 = Oracle(P, 62)
    cfg = BT.BootConfig(o0, w, w0, C)
    s_pt = (cfg.delta0 * float(P.q[1])) / P.delta[1]
    m = P.n // 2
    plans = [[o0.conv_plan(W[C * j:C * (j + 1), C * i:C * (i + 1)], C, C, 3, w, 1, s_pt) for i in range(2)]
             for j in range(2)]
    rots = sorted(set().union(*[set(p.rotations(m)) for row in plans for p in row]) |
                  set(BT.block_rotations(o0, None, cfg)))
    K, o, ctx, keys = make_pair("cfg2_small", 62, rotations=rots)
    cfg = BT.BootConfig(o, w, w0, C)
    pts = [o.encode_pt(E.cins_input_slots(x[C * i:C * (i + 1)], w, P.n), 1, P.delta[1]) for i in range(2)]
    cts = [o.encrypt(pt, 3 + i) for i, pt in enumerate(pts)]
    gcts = [K.ckks_encrypt(ctx, keys, import_pt(K, ctx, pt), 3 + i) for i, pt in enumerate(pts)]
    bt = K.ckks_boot_create(ctx, w, w0, C)
    _import_boot(K, ctx, bt, cfg)
    want = BT.block_multi(o, cts, plans[0], cfg)
    got = K.ckks_block_multi(ctx, keys, gcts, [import_plan(K, ctx, p) for p in plans[0]], bt)
    assert_ct_equal(K, ctx, got, want, "stage layer, output ciphertext 0")
    bt2 = K.ckks_boot_create(ctx, w, w0, C)
    ref = E.conv2d_same(x, W)
    for j in range(2):
        sets = [K.ckks_ptset_conv_fused(ctx, W[C * j:C * (j + 1), C * i:C * (i + 1)], C, C, 3, w, 1, s_pt)
                for i in range(2)]
        for ps in sets:
            K.ckks_keys_add_rotations(ctx, keys, K.ckks_ptset_rotations(ps))
        K.ckks_keys_add_rotations(ctx, keys, K.ckks_boot_rotations(bt2))
        out = K.ckks_block_multi(ctx, keys, gcts, sets, bt2)
        want_j = np.stack([E.flatten_padded(v, w) for v in ref[C * j:C * (j + 1)]])
        assert np.abs(_slots_pixels(K, ctx, keys, out, w, C) - want_j).max() < 2.0 ** -12
