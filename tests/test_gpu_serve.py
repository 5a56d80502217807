"""Serving loop on the GPU: continuous batching over slots, HBM-budget admission, p50/p99,
results identical alone and in a Poisson mix, host-side faults leave the loop serving."""
import time

import numpy as np
import pytest

import workloads as WL
from oracle import encoding as E
from tests.pairs import gpu_ctx

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def env():
    """config-2 chain at N = 2^10: one conv2d + bootstrap block (model A) and a chain of two
    blocks (model B), on a context created on its own stream"""
    from paper_2312_04356_gb300 import ckks as K
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gpu_ctx("cfg2_small", 71)
    spec = WL.CONV["cfg2_small"]
    w = E.pad_width(spec["w0"], spec["f"])
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    bt = K.ckks_boot_create(ctx, w, spec["w0"], spec["cout"])
    W = WL.weights(71, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    conv = K.ckks_ptset_conv_fused(ctx, W, spec["cin"], spec["cout"], spec["f"], w, 1, (2.0 ** 49 * q[1]) / delta[1])
    rots = sorted(set(K.ckks_ptset_rotations(conv)) | set(K.ckks_boot_rotations(bt)))
    keys = K.ckks_keygen(ctx, rots, True)

    def make_input(seed):
        x = WL.image(seed, spec["cin"], spec["w0"])
        ct = K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, x, w, 1, delta[1]), seed)
        return x, K.ckks_ct_export_rns(ctx, ct)

    def eager(limbs, n_blocks):
        ct = K.ckks_ct_import_rns(ctx, limbs, 1, delta[1])
        for b in range(n_blocks):
            if b:
                ct = K.ckks_level_down(ctx, ct, 1)
            ct = K.ckks_block(ctx, keys, ct, conv, bt)
        return K.ckks_ct_export_rns(ctx, ct)

    return dict(K=K, ctx=ctx, keys=keys, bt=bt, conv=conv, W=W, w=w, spec=spec, delta=delta, rots=rots,
                make_input=make_input, eager=eager, stream=stream)


def _server(env, slots, budget=0):
    K = env["K"]
    srv = K.ckks_server_create(env["ctx"], env["keys"], slots, budget)
    a = K.ckks_server_add_model(srv, [env["conv"]], [env["bt"]])
    b = K.ckks_server_add_model(srv, [env["conv"], env["conv"]], [env["bt"], env["bt"]])
    return srv, a, b


def test_results_identical_alone_and_in_mix(env):
    """one request alone, then the same input inside a Poisson mix of 70% one-block and 30%
    two-block requests on 4 slots: bit-identical results, equal to the eager C-ABI path;
    the one-block output decodes to FP64 conv2d within 2^-12"""
    K, ctx = env["K"], env["ctx"]
    n = ctx.n
    srv, A, B = _server(env, 4)
    info = K.ckks_server_model_info(srv, A)
    assert info["in_level"] == 1 and info["footprint"] > 0 and info["kernels"] > 100
    K.ckks_server_start(srv)
    x0, limbs0 = env["make_input"](1)
    rid = K.ckks_server_submit(srv, A, limbs0, 1, env["delta"][1])
    assert K.ckks_server_wait(srv, rid, 60) == K.CKKS_REQ_DONE
    alone, lev, sc = K.ckks_server_result(srv, rid, n)
    assert (alone == env["eager"](limbs0, 1)).all()
    got = K.ckks_decode_image(ctx, K.ckks_decrypt(ctx, env["keys"], K.ckks_ct_import_rns(ctx, alone, lev, sc)),
                              env["spec"]["cout"], env["spec"]["w0"], env["w"])
    assert np.abs(got - E.conv2d_same(x0, env["W"])[: env["spec"]["cout"]]).max() < 2.0 ** -12

    g = np.random.default_rng(5)
    inputs = {s: env["make_input"](s)[1] for s in range(2, 8)}
    mix = []
    for i in range(24):
        model = A if g.random() < 0.7 else B
        seed = 1 if i == 11 else int(g.integers(2, 8))
        lim = limbs0 if seed == 1 else inputs[seed]
        mix.append((K.ckks_server_submit(srv, model, lim, 1, env["delta"][1]), model, seed))
        time.sleep(float(g.exponential(0.002)))
    for rid, model, seed in mix:
        assert K.ckks_server_wait(srv, rid, 120) == K.CKKS_REQ_DONE
    refs = {}
    for rid, model, seed in mix:
        out, _, _ = K.ckks_server_result(srv, rid, n)
        if seed == 1 and model == A:
            assert (out == alone).all()
        key = (model, seed)
        if key not in refs:
            refs[key] = env["eager"](limbs0 if seed == 1 else inputs[seed], 1 if model == A else 2)
        assert (out == refs[key]).all()
    st = K.ckks_server_stats(srv)
    assert st["completed"] == 25 and st["failed"] == 0
    assert st["max_in_flight"] >= 2 and 0 < st["p50_ms"] <= st["p99_ms"]
    srv.close()


def test_budget_admission(env):
    """an HBM budget below two requests' temporaries keeps one request in flight on 4 slots;
    without a budget several run at once"""
    K = env["K"]
    srv, A, B = _server(env, 4)
    fp = K.ckks_server_model_info(srv, A)["footprint"]
    srv.close()
    _, limbs = env["make_input"](3)
    for budget, want_max in ((int(1.5 * fp), 1), (0, None)):
        srv = K.ckks_server_create(env["ctx"], env["keys"], 4, budget)
        A = K.ckks_server_add_model(srv, [env["conv"]], [env["bt"]])
        K.ckks_server_start(srv)
        ids = [K.ckks_server_submit(srv, A, limbs, 1, env["delta"][1]) for _ in range(8)]
        assert all(K.ckks_server_wait(srv, r, 120) == K.CKKS_REQ_DONE for r in ids)
        st = K.ckks_server_stats(srv)
        if want_max is not None:
            assert st["max_in_flight"] == want_max
        else:
            assert st["max_in_flight"] >= 2
        srv.close()


def test_faults_leave_the_loop_serving(env):
    """host-side faults: a model needing an absent key (CKKS_ENOKEY), a model above the budget
    (CKKS_ENOMEM), a request at the wrong level (CKKS_EINVAL), a cancelled queued request;
    the server keeps serving the others"""
    K, ctx = env["K"], env["ctx"]
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    # keys without one rotation that the conv needs: the model cannot be added
    need = K.ckks_ptset_rotations(env["conv"])
    short = K.ckks_keygen(ctx, [r for r in env["rots"] if r != need[-1]], True)
    srv_short = K.ckks_server_create(ctx, short, 1, 0)
    with pytest.raises(K.CkksError) as ei:
        K.ckks_server_add_model(srv_short, [env["conv"]], [env["bt"]])
    assert ei.value.code == K.CKKS_ENOKEY
    srv_short.close()
    srv = K.ckks_server_create(ctx, env["keys"], 1, 0)
    A = K.ckks_server_add_model(srv, [env["conv"]], [env["bt"]])
    K.ckks_server_start(srv)
    _, limbs = env["make_input"](4)
    with pytest.raises(K.CkksError) as ei:
        K.ckks_server_submit(srv, A, limbs, 2, delta[1])
    assert ei.value.code == K.CKKS_EINVAL
    ids = [K.ckks_server_submit(srv, A, limbs, 1, delta[1]) for _ in range(4)]
    K.ckks_server_cancel(srv, ids[3])          # one slot: the last one is still queued
    states = [K.ckks_server_wait(srv, r, 120) for r in ids]
    assert states[:3] == [K.CKKS_REQ_DONE] * 3 and states[3] == K.CKKS_REQ_CANCELLED
    ref = env["eager"](limbs, 1)
    for r in ids[:3]:
        assert (K.ckks_server_result(srv, r, ctx.n)[0] == ref).all()
    st = K.ckks_server_stats(srv)
    assert st["completed"] == 3 and st["cancelled"] == 1
    srv.close()
    tiny = K.ckks_server_create(ctx, env["keys"], 1, 1024)
    with pytest.raises(K.CkksError) as ei:
        K.ckks_server_add_model(tiny, [env["conv"]], [env["bt"]])
    assert ei.value.code == K.CKKS_ENOMEM
    tiny.close()


def test_block_batch_equals_blocks_alone(env):
    """ckks_block_batch_create / ckks_batch_launch: 5 inputs round-robin over 2 streams,
    launched twice; every output equals the eager block of its input; an output that aliases
    an input is refused before anything is recorded"""
    K, ctx = env["K"], env["ctx"]
    ins, want = [], []
    for i in range(5):
        _, limbs = env["make_input"](300 + i)
        ins.append(K.ckks_ct_import_rns(ctx, limbs, 1, env["delta"][1]))
        want.append(env["eager"](limbs, 1))
    outs = [K.ckks_ct_create(ctx) for _ in ins]
    with pytest.raises(K.CkksError) as ei:
        K.ckks_block_batch_create(ctx, env["keys"], ins, env["conv"], env["bt"], [ins[0]] + outs[1:], 2)
    assert ei.value.code == K.CKKS_EINVAL
    batch = K.ckks_block_batch_create(ctx, env["keys"], ins, env["conv"], env["bt"], outs, 2)
    for _ in range(2):
        K.ckks_batch_launch(batch)
        K.ckks_sync(ctx)
        for o, w in zip(outs, want):
            assert (K.ckks_ct_export_rns(ctx, o) == w).all()
    batch.close()


@pytest.mark.slow
def test_full_size_results_identical_alone_and_in_mix():
    """config 2 at full size (N = 2^16, 24 limbs): one request alone, then the same input among
    ten 1- and 2-block requests arriving together on 4 slots: bit-identical results, equal to
    the eager C-ABI path, the one-block output within 2^-12 of FP64 conv2d"""
    from paper_2312_04356_gb300 import ckks as K
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gpu_ctx("cfg2", 72)
    spec = WL.CONV["cfg2"]
    w = E.pad_width(spec["w0"], spec["f"])
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    bt = K.ckks_boot_create(ctx, w, spec["w0"], spec["cout"])
    W = WL.weights(72, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    conv = K.ckks_ptset_conv_fused(ctx, W, spec["cin"], spec["cout"], spec["f"], w, 1, (2.0 ** 49 * q[1]) / delta[1])
    keys = K.ckks_keygen(ctx, sorted(set(K.ckks_ptset_rotations(conv)) | set(K.ckks_boot_rotations(bt))), True)
    xs = {s: WL.image(s, spec["cin"], spec["w0"]) for s in range(1, 5)}
    limbs = {s: K.ckks_ct_export_rns(ctx, K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, x, w, 1, delta[1]), s))
             for s, x in xs.items()}

    def eager(lim, n_blocks):
        ct = K.ckks_ct_import_rns(ctx, lim, 1, delta[1])
        for b in range(n_blocks):
            if b:
                ct = K.ckks_level_down(ctx, ct, 1)
            ct = K.ckks_block(ctx, keys, ct, conv, bt)
        return K.ckks_ct_export_rns(ctx, ct)

    srv = K.ckks_server_create(ctx, keys, 4, 0)
    A = K.ckks_server_add_model(srv, [conv], [bt])
    B = K.ckks_server_add_model(srv, [conv, conv], [bt, bt])
    K.ckks_server_start(srv)
    rid = K.ckks_server_submit(srv, A, limbs[1], 1, delta[1])
    assert K.ckks_server_wait(srv, rid, 120) == K.CKKS_REQ_DONE
    alone, lev, sc = K.ckks_server_result(srv, rid, ctx.n)
    assert (alone == eager(limbs[1], 1)).all()
    got = K.ckks_decode_image(ctx, K.ckks_decrypt(ctx, keys, K.ckks_ct_import_rns(ctx, alone, lev, sc)),
                              spec["cout"], spec["w0"], w)
    assert np.abs(got - E.conv2d_same(xs[1], W)[: spec["cout"]]).max() < 2.0 ** -12
    plan = [(A, 2), (B, 3), (A, 1), (A, 4), (B, 1), (A, 3), (A, 2), (B, 4), (A, 1), (A, 4)]
    ids = [(K.ckks_server_submit(srv, m, limbs[s], 1, delta[1]), m, s) for m, s in plan]
    refs = {}
    for r, m, s in ids:
        assert K.ckks_server_wait(srv, r, 300) == K.CKKS_REQ_DONE
        out, _, _ = K.ckks_server_result(srv, r, ctx.n)
        if (m, s) not in refs:
            refs[(m, s)] = alone if (m, s) == (A, 1) else eager(limbs[s], 1 if m == A else 2)
        assert (out == refs[(m, s)]).all()
    st = K.ckks_server_stats(srv)
    assert st["completed"] == 11 and st["failed"] == 0 and st["max_in_flight"] >= 2
    srv.close()
