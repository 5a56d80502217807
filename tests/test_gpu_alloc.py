"""Device memory from a caller-provided allocator (ckks_ctx_set_allocator): the Alg. 1 block
at N = 2^10 with every buffer served by PyTorch's caching allocator is bit-exact against the
oracle, takes nothing from the library's own stream-ordered pool, and gives every byte back."""
import numpy as np
import pytest

import workloads as WL
from oracle import boot as BT
from oracle import encoding as E
from oracle.scheme import Oracle
from tests.pairs import assert_ct_equal, gpu_ctx, import_plan, import_pt, oracle_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()


def test_block_on_the_torch_allocator_bitexact():
    from paper_2312_04356_gb300 import ckks as K
    name, seed = "cfg2_small", 36
    P = oracle_params(name)
    spec = WL.CONV[name]
    x = WL.image(seed, spec["cin"], spec["w0"])
    W = WL.weights(seed, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    w = E.pad_width(spec["w0"], spec["f"])
    o = Oracle(P, seed)
    cfg = BT.BootConfig(o, w, spec["w0"], spec["cout"])
    plan = o.conv_plan(W, spec["cin"], spec["cout"], spec["f"], w, 1, (cfg.delta0 * float(P.q[1])) / P.delta[1])
    rots = BT.block_rotations(o, plan, cfg)
    o.gen_relin_key()
    o.gen_conj_key()
    o.gen_rotation_keys(rots)
    pt = o.encode_pt(E.cins_input_slots(x, w, P.n), 1, P.delta[1])
    want = BT.block(o, o.encrypt(pt, 2), plan, cfg)

    torch.cuda.synchronize()
    torch_base = torch.cuda.memory_allocated()
    calls = {"alloc": 0, "free": 0, "bytes": 0}
    t_alloc, t_free = K.torch_allocator()

    def alloc(nbytes, stream):
        calls["alloc"] += 1
        calls["bytes"] += nbytes
        return t_alloc(nbytes, stream)

    def free(ptr, nbytes, stream):
        calls["free"] += 1
        t_free(ptr, nbytes, stream)

    ctx = gpu_ctx(name, seed)
    K.ckks_ctx_set_allocator(ctx, alloc, free)
    pool0 = K.ckks_ctx_pool_stats(ctx, reset_high=True)
    keys = K.ckks_keygen(ctx, rots, True)
    bt = K.ckks_boot_create(ctx, w, spec["w0"], spec["cout"])
    for i, p in enumerate(cfg.ctos):
        K.ckks_boot_set_ctos(ctx, bt, i, import_plan(K, ctx, p))
    for i, p in enumerate(cfg.stoc):
        K.ckks_boot_set_stoc(ctx, bt, i, import_plan(K, ctx, p))
    K.ckks_boot_set_coeffs(ctx, bt, cfg.coeffs)
    K.ckks_boot_set_masks(ctx, bt, import_pt(K, ctx, cfg.pt_mask_re), import_pt(K, ctx, cfg.pt_mask_im))
    gct = K.ckks_encrypt(ctx, keys, import_pt(K, ctx, pt), 2)
    out = K.ckks_block(ctx, keys, gct, import_plan(K, ctx, plan), bt)
    assert_ct_equal(K, ctx, out, want, "block on the caller allocator")
    pool1 = K.ckks_ctx_pool_stats(ctx)
    # every buffer came from the caller allocator: the pool never held more than before
    assert pool1["used_high"] == pool0["used"], (pool0, pool1)
    assert calls["alloc"] > 100 and torch.cuda.memory_allocated() > torch_base
    del out, gct, keys, bt
    import gc
    gc.collect()
    torch.cuda.synchronize()
    assert calls["free"] == calls["alloc"]
    assert torch.cuda.memory_allocated() == torch_base


def test_allocator_arguments():
    from paper_2312_04356_gb300 import ckks as K
    ctx = gpu_ctx("cfg1", 3)
    with pytest.raises(ValueError):
        K.ckks_ctx_set_allocator(ctx, alloc=lambda n, s: 0)
    calls = {"n": 0}

    def failing(nbytes, stream):
        calls["n"] += 1
        return 0
    K.ckks_ctx_set_allocator(ctx, failing, lambda p, n, s: None)
    with pytest.raises(K.CkksError) as e:
        K.ckks_keygen(ctx, [1], False)
    assert e.value.code == K.CKKS_ENOMEM and calls["n"] >= 1
    K.ckks_ctx_set_allocator(ctx)                          # back to the library's pool
    keys = K.ckks_keygen(ctx, [1], False)
    z = WL.slots(1, ctx.n // 2)
    _, _, _, delta = K.ckks_ctx_info(ctx)
    ct = K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, z, 3, delta[3]), 1)
    assert np.abs(K.ckks_decode(ctx, K.ckks_decrypt(ctx, keys, ct)) - z).max() < 1e-6
