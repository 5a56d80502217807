"""The allocation-free rescale (ckks_rescale_noalloc) against ckks_rescale.

Callers that cannot allocate device memory mid-run (graphs recorded without pool nodes,
serving loops that forbid cudaMalloc) use ckks_rescale_noalloc, whose scratch is a static
device array.  Its output must be identical to ckks_rescale's, on consecutive calls that
reuse the same scratch, and it must take no memory from any allocator.  This file is
collected last on purpose.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as WL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _setup(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()
    from paper_2312_04356_gb300 import ckks as K
    return K, K.ckks_ctx_create(WL.PARAMS[name], 5, torch.cuda.current_stream().cuda_stream)


def _input(K, ctx, q, level, seed):
    """a ciphertext at `level` as device NTT-domain limbs, and ckks_rescale's output for it
    (coefficient domain; any residues will do: the rescale is exact)"""
    n = ctx.n
    ids = list(range(level + 1)) * 2
    host = WL.residues(seed, [q[i] for i in ids], n).reshape(2, level + 1, n)
    want = K.ckks_ct_export_rns(ctx, K.ckks_rescale(ctx, K.ckks_ct_import_rns(ctx, host, level, 2.0 ** 40)))
    d_in = torch.from_numpy(host.reshape(-1).view(np.int64).copy()).cuda()
    K.ckks_ntt_forward(ctx, d_in.data_ptr(), 2 * (level + 1), ids)
    return d_in, want


def _read(K, ctx, d_out, level):
    K.ckks_ntt_inverse(ctx, d_out.data_ptr(), 2 * level, list(range(level)) * 2)
    torch.cuda.synchronize()
    return d_out.cpu().numpy().view(np.uint64).reshape(2, level, ctx.n)


def test_first_call_inside_a_capture_is_refused():
    """in a fresh process, a first call on a capturing stream (where the scratch address could
    not be looked up) returns CKKS_EINVAL and enqueues nothing; the same call outside the
    capture then works"""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()
    code = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import workloads as WL
from paper_2312_04356_gb300 import ckks as K
s = torch.cuda.Stream()
with torch.cuda.stream(s):
    ctx = K.ckks_ctx_create(WL.PARAMS["cfg1"], 5, s.cuda_stream)
    buf = torch.zeros(2 * 4 * ctx.n, dtype=torch.int64, device="cuda")
    out = torch.zeros(2 * 3 * ctx.n, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    code = 0
    g.capture_begin()
    try:
        K.ckks_rescale_noalloc(ctx, buf.data_ptr(), 3, out.data_ptr())
    except K.CkksError as e:
        code = e.code
    g.capture_end()
    assert code == K.CKKS_EINVAL, code
    K.ckks_rescale_noalloc(ctx, buf.data_ptr(), 3, out.data_ptr())
    torch.cuda.synchronize()
print("refused-in-capture-ok")
""" % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "refused-in-capture-ok" in r.stdout, r.stdout + r.stderr


@pytest.mark.parametrize("name,level", [("cfg1", 3), ("cfg1", 1), ("cfg2", 23), ("cfg2", 5)])
def test_rescale_noalloc_matches_rescale(name, level):
    K, ctx = _setup(name)
    q, _, _, _ = K.ckks_ctx_info(ctx)
    for call in range(2):
        d_in, want = _input(K, ctx, q, level, 100 + call)
        d_out = torch.zeros(2 * level * ctx.n, dtype=torch.int64, device="cuda")
        K.ckks_rescale_noalloc(ctx, d_in.data_ptr(), level, d_out.data_ptr())
        assert (_read(K, ctx, d_out, level) == want).all(), "call %d differs" % call


def test_back_to_back_calls_share_the_scratch_in_stream_order():
    """two calls on the same stream with different inputs and outputs and no synchronisation
    between them: the second reuses the scratch after the first in stream order, and both
    outputs equal ckks_rescale's"""
    K, ctx = _setup("cfg2")
    q, _, _, _ = K.ckks_ctx_info(ctx)
    level = 17
    (a, wa), (b, wb) = _input(K, ctx, q, level, 7), _input(K, ctx, q, level, 8)
    torch.cuda.synchronize()
    oa = torch.zeros(2 * level * ctx.n, dtype=torch.int64, device="cuda")
    ob = torch.zeros_like(oa)
    K.ckks_rescale_noalloc(ctx, a.data_ptr(), level, oa.data_ptr())
    K.ckks_rescale_noalloc(ctx, b.data_ptr(), level, ob.data_ptr())
    assert (_read(K, ctx, oa, level) == wa).all()
    assert (_read(K, ctx, ob, level) == wb).all()


def test_rescale_noalloc_takes_no_memory():
    """with a counting caller allocator installed and the pool's high-water mark reset, the
    call takes nothing from either (ckks_rescale on the same context does, through the
    caller allocator: the check would see a temporary buffer)"""
    K, ctx = _setup("cfg2")
    q, _, _, _ = K.ckks_ctx_info(ctx)
    level = 23
    d_in, want = _input(K, ctx, q, level, 9)
    d_out = torch.zeros(2 * level * ctx.n, dtype=torch.int64, device="cuda")
    calls = {"alloc": 0, "free": 0}
    t_alloc, t_free = K.torch_allocator()

    def alloc(nbytes, stream):
        calls["alloc"] += 1
        return t_alloc(nbytes, stream)

    def free(ptr, nbytes, stream):
        calls["free"] += 1
        t_free(ptr, nbytes, stream)
    K.ckks_ctx_set_allocator(ctx, alloc, free)
    before = K.ckks_ctx_pool_stats(ctx, reset_high=True)
    torch_before = torch.cuda.memory_allocated()
    K.ckks_rescale_noalloc(ctx, d_in.data_ptr(), level, d_out.data_ptr())
    after = K.ckks_ctx_pool_stats(ctx)
    assert calls == {"alloc": 0, "free": 0}
    assert after["used_high"] == before["used"] and after["used"] == before["used"]
    assert torch.cuda.memory_allocated() == torch_before
    assert (_read(K, ctx, d_out, level) == want).all()
    ct = K.ckks_ct_import_rns(ctx, np.zeros((2, level + 1, ctx.n), dtype=np.uint64), level, 2.0 ** 40)
    K.ckks_rescale(ctx, ct)
    assert calls["alloc"] > 0
    K.ckks_ctx_set_allocator(ctx)


def test_rescale_noalloc_rejects_bad_arguments():
    K, ctx = _setup("cfg1")
    buf = torch.zeros(2 * 4 * ctx.n, dtype=torch.int64, device="cuda")
    with pytest.raises(K.CkksError):
        K.ckks_rescale_noalloc(ctx, buf.data_ptr(), 0, buf.data_ptr())       # level 0 cannot rescale
    with pytest.raises(K.CkksError):
        K.ckks_rescale_noalloc(ctx, buf.data_ptr(), 3, buf.data_ptr())       # overlapping in / out


def test_rescale_noalloc_rejects_sizes_above_the_array():
    """N = 2^17 with 17 limbs at level 16 needs (2 * 16 + 2) 2^17 > 2^22 scratch words: refused
    with CKKS_EINVAL before any device work (the small buffers are never touched)"""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()
    from paper_2312_04356_gb300 import ckks as K
    params = dict(log_n=17, n_q=17, dnum=2, n_p=0, q0_bits=60, scale_bits=40, p_bits=60, boot_bits=0, n_boot=0,
                  h=0, sigma=3.2)
    ctx = K.ckks_ctx_create(params, 5, torch.cuda.current_stream().cuda_stream)
    a = torch.zeros(16, dtype=torch.int64, device="cuda")
    b = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(K.CkksError) as e:
        K.ckks_rescale_noalloc(ctx, a.data_ptr(), 16, b.data_ptr())
    assert e.value.code == K.CKKS_EINVAL and "scratch" in str(e.value)
