"""Edge cases and error returns of the C ABI on the GPU: degenerate inputs give clean error
codes (no fault, the context stays usable); the largest supported ring N = 2^17 and the
smallest N = 2^3 still compute bit-exact NTTs; ragged and empty shapes behave."""
import numpy as np
import pytest

import workloads as WL
from oracle import encoding as E
from tests.pairs import assert_ct_equal, gpu_ctx, import_ct, make_pair

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()


def _code(K, fn):
    with pytest.raises(K.CkksError) as ei:
        fn()
    return ei.value.code


def test_error_returns_leave_the_context_usable():
    K, o, ctx, keys = make_pair("cfg1", 91, rotations=[1])
    P = o.P
    z = WL.slots(91, P.n // 2, 0.5)
    ct = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, z, 1, P.delta[1]), 1)
    c0 = K.ckks_rescale(ctx, ct)                              # level 0
    assert _code(K, lambda: K.ckks_rescale(ctx, c0)) == K.CKKS_ELEVEL
    hi = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, z, P.L, P.delta[P.L]), 2)
    assert _code(K, lambda: K.ckks_add(ctx, ct, hi)) == K.CKKS_EINVAL          # level mismatch
    assert _code(K, lambda: K.ckks_rotate_hoisted(ctx, keys, hi, [2])) == K.CKKS_ENOKEY
    assert _code(K, lambda: K.ckks_encode(ctx, np.full(P.n // 2, 1e12), P.L, P.delta[P.L])) == K.CKKS_EINVAL
    assert _code(K, lambda: K.ckks_ctx_set_ntt_variant(ctx, 7)) == K.CKKS_EINVAL
    empty = K.ckks_ptset_create(ctx, 0, 1, 4, 2, P.L, P.delta[P.L])
    assert _code(K, lambda: K.ckks_bsgs(ctx, keys, hi, empty)) == K.CKKS_EINVAL
    assert _code(K, lambda: K.ckks_ct_import_rns(ctx, np.zeros((2, P.L + 2, P.n), dtype=np.uint64), P.L + 1, 1.0)
                 ) == K.CKKS_EINVAL
    # downsampling depthwise sets (w_in = 8: C = N / 64 channels per input ciphertext)
    C = P.n // 64
    dw = K.ckks_ptset_dwconv_fused_s2
    assert _code(K, lambda: dw(ctx, np.ones((4, 2, 2)), 8, 0, 1, 1.0)) == K.CKKS_EINVAL           # even kernel
    assert _code(K, lambda: dw(ctx, np.ones((4, 3, 3)), 8, 1, 1, 1.0)) == K.CKKS_EINVAL           # no channel in t = 1
    assert _code(K, lambda: dw(ctx, np.ones((4 * C + 1, 3, 3)), 8, 0, 1, 1.0)) == K.CKKS_EINVAL   # > 4C outputs
    # still usable: a rotation that has its key is bit-exact against the oracle
    oct_ = o.encrypt(o.encode_pt(z, P.L, P.delta[P.L]), 3)
    assert_ct_equal(K, ctx, K.ckks_rotate_hoisted(ctx, keys, import_ct(K, ctx, oct_), [1])[0], o.rotate(oct_, 1),
                    "rotation after errors")
    K.ckks_sync(ctx)


@pytest.mark.parametrize("log_n", [3, 17])
def test_ntt_extreme_ring_sizes_bitexact(log_n):
    """N = 2^3 (smallest) and N = 2^17 (largest supported): forward NTT bit-exact against the
    oracle's NTT and the inverse returns the input"""
    from oracle import _clib as C
    from oracle import params as PP
    from paper_2312_04356_gb300 import ckks as K
    d = dict(log_n=log_n, n_q=3, dnum=1, n_p=1, q0_bits=60, scale_bits=40 if log_n > 3 else 30, p_bits=60,
             boot_bits=0, n_boot=0, h=0, sigma=3.2)
    P = PP.Params(log_n, 3, 1, 60, d["scale_bits"], 60, h=0, n_p=1)
    ctx = K.ckks_ctx_create(d, 1, torch.cuda.current_stream().cuda_stream)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    assert q == list(P.q) and p == list(P.p)
    mods = q + p
    ids = list(range(len(mods)))
    x = WL.residues(5, mods, 1 << log_n)
    dev = torch.from_numpy(x.view(np.int64).copy()).cuda()
    K.ckks_ntt_forward(ctx, dev.data_ptr(), len(ids), ids)
    torch.cuda.synchronize()
    assert (dev.cpu().numpy().view(np.uint64) == C.ntt_forward(x, mods, list(P.psi_q) + list(P.psi_p), log_n)).all()
    K.ckks_ntt_inverse(ctx, dev.data_ptr(), len(ids), ids)
    torch.cuda.synchronize()
    assert (dev.cpu().numpy().view(np.uint64) == x).all()


def test_ragged_and_empty_shapes():
    """one channel of 16 x 16 in a 32-wide slice (3 of 4 slices empty), a 1x1 kernel and a
    kernel as wide as the image: fused conv decodes to FP64 conv2d; zero limbs to an NTT call
    are a no-op"""
    from paper_2312_04356_gb300 import ckks as K
    P_ = WL.PARAMS["cfg1"]
    ctx = gpu_ctx("cfg1", 92)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    L = len(q) - 1
    for f, w0 in ((1, 16), (15, 16)):
        w = E.pad_width(w0, f)
        x = WL.image(92 + f, 1, w0)
        W = WL.weights(92 + f, 1, 1, f, "uniform")
        conv = K.ckks_ptset_conv_fused(ctx, W, 1, 1, f, w, L, (delta[L - 1] * q[L]) / delta[L])
        keys = K.ckks_keygen(ctx, K.ckks_ptset_rotations(conv), False)
        ct = K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, x, w, L, delta[L]), 5)
        out = K.ckks_conv2d_cins(ctx, keys, ct, conv)
        coeffs = K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, out), K.CKKS_COEFF)
        got = E.conv_output_from_coeffs(coeffs, (1 << P_["log_n"]) // (w * w), w * w, 1, w, w0)
        assert np.abs(got - E.conv2d_same(x, W)).max() < 2.0 ** -12
    dev = torch.zeros(8, dtype=torch.int64, device="cuda")
    K.ckks_ntt_forward(ctx, dev.data_ptr(), 0, [])
    torch.cuda.synchronize()
