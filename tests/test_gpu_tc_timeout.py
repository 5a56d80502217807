"""The bounded waits of the tensor-core base conversion, exercised on the GPU without any fault:
a test hook withholds the conversion's MMAs, so that every CTA's wait on its MMA barrier runs
out after about a second; the kernel records the timeout, releases its tensor memory and
returns, ckks_sync reports CKKS_ETIMEOUT, and once the record is cleared the same context
computes the key switch bit-exactly again (config-2 chain at N = 2^10: eight tiles per limb,
so each withheld launch ends in about a second)."""
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


def test_withheld_mma_times_out_and_the_context_recovers():
    K, o, ctx, keys = make_pair("cfg2_small", 31, rotations=[1], conj=False)
    P = o.P
    lev = P.L
    ct = o.encrypt(o.encode_pt(WL.slots(3, P.n // 2, 0.4), lev, P.delta[lev]), 7)
    g = import_ct(K, ctx, ct)
    want = o.rotate(ct, 1)
    K.ckks_ctx_set_tensor_conversion(ctx, 1)
    K.ckks_sync(ctx)
    assert K.ckks_ctx_take_device_faults(ctx) == 0
    try:
        K.ckks_debug_withhold_tensor_commit(ctx, 1)
        K.ckks_rotate_hoisted(ctx, keys, g, [1])
        with pytest.raises(K.CkksError) as err:
            K.ckks_sync(ctx)
        assert err.value.code == K.CKKS_ETIMEOUT
    finally:
        K.ckks_debug_withhold_tensor_commit(ctx, 0)
        timeouts = K.ckks_ctx_take_device_faults(ctx)
    assert timeouts > 0
    K.ckks_sync(ctx)
    got = K.ckks_rotate_hoisted(ctx, keys, g, [1])[0]
    assert_ct_equal(K, ctx, got, want, "rotation after the timeouts")
    assert K.ckks_ctx_take_device_faults(ctx) == 0
