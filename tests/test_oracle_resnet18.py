"""Pins of the ImageNet-shaped (ResNet-18) layers on the oracle, at reduced N.

* The 7x7 stride-2 stem: the client encodes the polyphase images of its input directly (the
  first layer's input is a fresh client encoding, so Alg. 2's homomorphic decomposition is not
  needed there), one input channel per ciphertext; the decomposed kernels then give the
  stride-2 conv as a unit-stride conv (Alg. 2, App. B), checked in FP64 for f = 7 and f = 1 (the
  1x1 stride-2 shortcut) and under encryption against FP64 conv2d.
* A stage layer whose channels span several ciphertexts on both sides (Sec. 3.3.3, C_in, C_out
  > C): output ciphertext j is the block matrix-vector product over the input ciphertexts,
  checked under encryption against FP64 conv2d for every output ciphertext.
"""
import numpy as np
import pytest

from oracle import boot as BT
from oracle import encoding as E
from oracle.scheme import Oracle
from tests.pairs import oracle_params

rng = np.random.default_rng(18)


def _conv_stride2_loops(x, W):
    cin, h, _ = x.shape
    cout, _, f, _ = W.shape
    c = f // 2
    out = np.zeros((cout, h // 2, h // 2))
    for o in range(cout):
        for y in range(h // 2):
            for xx in range(h // 2):
                for i in range(cin):
                    for a in range(f):
                        for b in range(f):
                            r, col = 2 * y + a - c, 2 * xx + b - c
                            if 0 <= r < h and 0 <= col < h:
                                out[o, y, xx] += W[o, i, a, b] * x[i, r, col]
    return out


@pytest.mark.parametrize("f", [7, 1])
def test_stem_polyphase_with_one_channel_per_ciphertext(f):
    """three input channels, one per ciphertext (C = 1: its four polyphase images are the four
    slices): the unit-stride convs of the polyphase images with the decomposed kernels, summed
    over the three ciphertexts, equal the stride-2 conv2d (brute force, zero padding f // 2)"""
    x = rng.random((3, 12, 12))
    W = rng.normal(size=(4, 3, f, f))
    pp = E.decompose_images(x)
    acc = sum(E.conv2d_same(pp[4 * t:4 * (t + 1)], E.decompose_kernels(W, 1, t)) for t in range(3))
    assert E.decompose_kernels(W, 1, 0).shape[2] == 2 * ((f // 2 + 1) // 2) + 1
    assert np.abs(acc - _conv_stride2_loops(x, W)).max() < 1e-12


def _encrypt_slices(o, imgs, w, level):
    P = o.P
    return o.encrypt(o.encode_pt(E.cins_input_slots(imgs, w, P.n), level, P.delta[level]), len(imgs))


@pytest.fixture(scope="module")
def small_chain():
    P = oracle_params("cfg2_small")       # the config-2 chain at N = 2^10
    o = Oracle(P, 18)
    o.gen_relin_key()
    o.gen_conj_key()
    return o


def test_stem_under_encryption(small_chain):
    """the stem at N = 2^10: a 3 x 28 x 28 input as three client-encoded ciphertexts of its
    polyphase images (14 x 14 in slices of width 16, C = 4 slices), a 7 x 7 stride-2 conv to 4
    channels by the decomposed kernels (5 x 5), one BSGS per input ciphertext summed before the
    rescale; the coefficient-encoded output decodes to the FP64 stride-2 conv; then the bootstrap
    and StoC1 of the 14 x 14 block bring it back to slots within 2^-12"""
    o = small_chain
    P = o.P
    x = rng.random((3, 28, 28))
    W = rng.normal(0, 0.1, (4, 3, 7, 7))
    pp = E.decompose_images(x)
    w = E.pad_width(14, 5)
    assert w == 16 and P.n // (w * w) == 4
    cts = [_encrypt_slices(o, pp[4 * t:4 * (t + 1)], w, 1) for t in range(3)]
    cfg = BT.BootConfig(o, w, 14, 4)
    s_pt = (cfg.delta0 * float(P.q[1])) / P.delta[1]
    plans = [o.conv_plan(E.decompose_kernels(W, 1, t), 4, 4, 5, w, 1, s_pt) for t in range(3)]
    m = P.n // 2
    o.gen_rotation_keys(sorted(set().union(*[set(p.rotations(m)) for p in plans]) |
                               set(BT.block_rotations(o, None, cfg))))
    conv = o.bsgs_multi(cts, plans, rescale=True)
    want = E.conv2d_stride2(x, W)
    got = E.conv_output_from_coeffs(o.decode_coeffs(o.decrypt(conv)), 4, w * w, 4, w, 14)
    assert np.abs(got - want).max() < 1e-6
    out = BT.block_multi(o, cts, plans, cfg)
    slots = o.decode_slots(o.decrypt(out))
    ell = w * w // 2
    pix = np.stack([E.encode(slots[i * ell:(i + 1) * ell], w * w) for i in range(4)])
    ref = np.stack([E.flatten_padded(v, w) for v in want])
    assert np.abs(pix - ref).max() < 2.0 ** -12


def test_stage_layer_spanning_ciphertexts(small_chain):
    """32 channels of 4 x 4 in two ciphertexts (w = 8, C = 16) -> 32 output channels in two
    ciphertexts: output ciphertext j sums the BSGS convs of both inputs with the weight blocks
    W[16 j : 16 j + 16, 16 i : 16 i + 16] (Sec. 3.3.3); every output decodes to FP64 conv2d"""
    o = small_chain
    P = o.P
    w0, w, C = 4, 8, 16
    x = rng.random((2 * C, w0, w0))
    W = rng.normal(0, 0.1, (2 * C, 2 * C, 3, 3))
    cts = [_encrypt_slices(o, x[C * i:C * (i + 1)], w, 1) for i in range(2)]
    s_pt = (2.0 ** 49 * float(P.q[1])) / P.delta[1]
    want = E.conv2d_same(x, W)
    m = P.n // 2
    for j in range(2):
        plans = [o.conv_plan(W[C * j:C * (j + 1), C * i:C * (i + 1)], C, C, 3, w, 1, s_pt) for i in range(2)]
        o.gen_rotation_keys(sorted(set(plans[0].rotations(m)) | set(plans[1].rotations(m))))
        out = o.bsgs_multi(cts, plans, rescale=True)
        got = E.conv_output_from_coeffs(o.decode_coeffs(o.decrypt(out)), C, w * w, C, w, w0)
        assert np.abs(got - want[C * j:C * (j + 1)]).max() < 1e-6
