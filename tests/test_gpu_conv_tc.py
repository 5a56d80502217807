"""Base conversion on the tensor cores (8-bit chunks, FP16 x FP16 -> FP32 MMAs in tensor memory)
against the integer-pipe kernel and the oracle: every key switch (ModUp of each digit, ModDown)
bit-exact at N = 2^16 on the config-2 chain, at levels whose digits have 8, 5, 3 and 1 limbs
(odd input counts are padded with a zero input; output groups of 12 or fewer), with either
kernel (one or two threads per coefficient row on the tensor cores, or the integer pipe); the
whole small block (ModDown fused with the exact rescale in every HMult) bit-exact with each;
and no bounded wait inside the kernel ever runs out."""
import numpy as np
import pytest

import workloads as WL
from tests.pairs import assert_ct_equal, import_ct, make_pair

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def full_pair():
    return make_pair("cfg2", 21, rotations=[1, 5])


@pytest.mark.parametrize("lev", [23, 20, 10, 2])
def test_key_switching_with_both_conversion_kernels(full_pair, lev):
    K, o, ctx, keys = full_pair
    P = o.P
    z = WL.slots(30 + lev, P.n // 2, 0.4)
    ct = o.encrypt(o.encode_pt(z, lev, P.delta[lev]), 40 + lev)
    g = import_ct(K, ctx, ct)
    want_rot = o.rotate_hoisted(ct, [1, 5])
    want_hm = o.mul_relin(ct, ct)
    want_cj = o.conjugate(ct)
    for tc in (2, 0, 1):
        K.ckks_ctx_set_tensor_conversion(ctx, tc)
        for s, gr, w in zip((1, 5), K.ckks_rotate_hoisted(ctx, keys, g, [1, 5]), want_rot):
            assert_ct_equal(K, ctx, gr, w, "level %d, rotation %d, tensor cores %d" % (lev, s, tc))
        assert_ct_equal(K, ctx, K.ckks_mul_relin(ctx, keys, g, g), want_hm, "level %d, HMult, tc %d" % (lev, tc))
        assert_ct_equal(K, ctx, K.ckks_conjugate(ctx, keys, g), want_cj, "level %d, conj, tc %d" % (lev, tc))
    K.ckks_ctx_set_tensor_conversion(ctx, 1)
    assert K.ckks_ctx_take_device_faults(ctx) == 0


def test_small_block_with_both_conversion_kernels():
    """the config-2 chain at N = 2^10 (8 tiles of 128 coefficients per limb): the whole block
    against the oracle with each kernel"""
    from tests.test_gpu_parity import _block_pair
    from oracle import boot as BT
    from tests.pairs import import_plan, import_pt
    d = _block_pair("cfg2_small", 5)
    K, o, ctx, keys = d["K"], d["o"], d["ctx"], d["keys"]
    ct = o.encrypt(d["pt"], 3)
    want = BT.block(o, ct, d["plan"], d["cfg"])
    gct = K.ckks_encrypt(ctx, keys, import_pt(K, ctx, d["pt"]), 3)
    gplan = import_plan(K, ctx, d["plan"])
    for tc in (2, 0, 1):
        K.ckks_ctx_set_tensor_conversion(ctx, tc)
        assert_ct_equal(K, ctx, K.ckks_block(ctx, keys, gct, gplan, d["bt"]), want, "block, tc %d" % tc)
    assert K.ckks_ctx_take_device_faults(ctx) == 0


def test_mode_outside_range_is_refused(full_pair):
    K, o, ctx, keys = full_pair
    for bad in (3, -1):
        with pytest.raises(K.CkksError):
            K.ckks_ctx_set_tensor_conversion(ctx, bad)
    K.ckks_ctx_set_tensor_conversion(ctx, 1)
