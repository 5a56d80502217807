"""The allocation-free rescale (ckks_rescale_noalloc) against ckks_rescale.

Callers that cannot allocate device memory mid-run (graphs recorded without pool nodes,
serving loops that forbid cudaMalloc) use ckks_rescale_noalloc, whose scratch is a static
device array.  Its output must be identical to ckks_rescale's, on consecutive calls that
reuse the same scratch.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as WL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("name,level", [("cfg1", 3), ("cfg1", 1), ("cfg2", 23), ("cfg2", 5)])
def test_rescale_noalloc_matches_rescale(name, level):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()
    from paper_2312_04356_gb300 import ckks as K
    ctx = K.ckks_ctx_create(WL.PARAMS[name], 5, torch.cuda.current_stream().cuda_stream)
    q, _, _, _ = K.ckks_ctx_info(ctx)
    n = ctx.n
    ids = list(range(level + 1)) * 2
    for call in range(2):
        # coefficient-domain residues of a ciphertext at `level` (any residues: rescale is exact)
        host = WL.residues(100 + call, [q[i] for i in ids], n).reshape(2, level + 1, n)
        want_ct = K.ckks_rescale(ctx, K.ckks_ct_import_rns(ctx, host, level, 2.0 ** 40))
        want = K.ckks_ct_export_rns(ctx, want_ct)
        d_in = torch.from_numpy(host.reshape(-1).view(np.int64).copy()).cuda()
        K.ckks_ntt_forward(ctx, d_in.data_ptr(), 2 * (level + 1), ids)
        d_out = torch.zeros(2 * level * n, dtype=torch.int64, device="cuda")
        K.ckks_rescale_noalloc(ctx, d_in.data_ptr(), level, d_out.data_ptr())
        K.ckks_ntt_inverse(ctx, d_out.data_ptr(), 2 * level, list(range(level)) * 2)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint64).reshape(2, level, n)
        assert (got == want).all(), "call %d differs" % call


def test_rescale_noalloc_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import ckks as K
    ctx = K.ckks_ctx_create(WL.PARAMS["cfg1"], 5, torch.cuda.current_stream().cuda_stream)
    buf = torch.zeros(2 * 4 * ctx.n, dtype=torch.int64, device="cuda")
    with pytest.raises(K.CkksError):
        K.ckks_rescale_noalloc(ctx, buf.data_ptr(), 0, buf.data_ptr())       # level 0 cannot rescale
    with pytest.raises(K.CkksError):
        K.ckks_rescale_noalloc(ctx, buf.data_ptr(), 3, buf.data_ptr())       # overlapping in / out
