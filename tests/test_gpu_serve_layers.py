"""Serving models made of layers over several ciphertexts (config-2 chain at N = 2^10): a block
layer with one input and two outputs followed by a Sec. 3.3.3 block over both, a ResNet-stage
pattern of a block whose EvalMod outputs feed an Alg. 2 downsampling layer and then a block of
the new shape, and layers whose outputs read chosen inputs.  Each request's result equals the same layers called eagerly
through the C ABI, limb for limb, alone and while the other model's requests run beside it."""
import numpy as np
import pytest

import workloads as WL
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
    from paper_2312_04356_gb300 import ckks as K
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gpu_ctx("cfg2_small", 83)
    q, _, _, delta = K.ckks_ctx_info(ctx)
    s_pt = (2.0 ** 49 * q[1]) / delta[1]
    C, w0, w = 16, 4, 8                       # 16 channels of 4 x 4 in slices of width 8
    rng = np.random.default_rng(83)

    def wts(cout, cin):
        return rng.normal(0.0, 0.1, (cout, cin, 3, 3))

    b1 = K.ckks_boot_create(ctx, w, w0, C)
    # model M1: one input -> two outputs (two blocks) -> one output over both (Sec. 3.3.3)
    m1_l1 = [[K.ckks_ptset_conv_fused(ctx, wts(C, C), C, C, 3, w, 1, s_pt)] for _ in range(2)]
    m1_l2 = [[K.ckks_ptset_conv_fused(ctx, wts(C, C), C, C, 3, w, 1, s_pt) for _ in range(2)]]
    # model M2: block -> its EvalMod outputs -> Alg. 2 to 64 channels of 2 x 2 (w = 4) -> block
    bt_in = K.ckks_boot_create(ctx, w, w0, C, stride=2)
    bt_out = K.ckks_boot_create(ctx, w // 2, w0 // 2, 4 * C)
    m2_l1 = [[K.ckks_ptset_conv_fused(ctx, wts(C, C), C, C, 3, w, 1, s_pt)]]
    m2_l2 = [[K.ckks_ptset_conv_fused_s2(ctx, wts(4 * C, C), C, 4 * C, 3, w, 0, 1, s_pt)]]
    m2_l3 = [[K.ckks_ptset_conv_fused(ctx, wts(4 * C, 4 * C), 4 * C, 4 * C, 3, w // 2, 1, s_pt)]]
    # model M3: outputs reading chosen inputs (the two ciphertexts swapped, one input each)
    m3_l1 = [[K.ckks_ptset_conv_fused(ctx, wts(C, C), C, C, 3, w, 1, s_pt)] for _ in range(2)]
    m3_l2 = [[K.ckks_ptset_conv_fused(ctx, wts(C, C), C, C, 3, w, 1, s_pt)] for _ in range(2)]
    m3_l3 = [[K.ckks_ptset_conv_fused(ctx, wts(C, C), C, C, 3, w, 1, s_pt) for _ in range(2)]]
    # model M4: two blocks' EvalMod outputs -> one Alg. 2 output from each -> one block over both
    m4_l1 = [[K.ckks_ptset_conv_fused(ctx, wts(C, C), C, C, 3, w, 1, s_pt)] for _ in range(2)]
    m4_l2 = [[K.ckks_ptset_conv_fused_s2(ctx, wts(4 * C, C), C, 4 * C, 3, w, 0, 1, s_pt)] for _ in range(2)]
    m4_l3 = [[K.ckks_ptset_conv_fused(ctx, wts(4 * C, 4 * C), 4 * C, 4 * C, 3, w // 2, 1, s_pt)
              for _ in range(2)]]
    sets = [p for L in (m1_l1, m1_l2, m2_l1, m2_l2, m2_l3, m3_l1, m3_l2, m3_l3, m4_l1, m4_l2, m4_l3)
            for row in L for p in row]
    rots = set()
    for p in sets:
        rots |= set(K.ckks_ptset_rotations(p))
    for b in (b1, bt_in, bt_out):
        rots |= set(K.ckks_boot_rotations(b))
    keys = K.ckks_keygen(ctx, sorted(rots), True)
    m1 = [dict(kind=K.CKKS_LAYER_BLOCK, convs=m1_l1, boot=b1), dict(kind=K.CKKS_LAYER_BLOCK, convs=m1_l2, boot=b1)]
    m2 = [dict(kind=K.CKKS_LAYER_BLOCK, convs=m2_l1, boot=bt_in),
          dict(kind=K.CKKS_LAYER_DOWNSAMPLE, convs=m2_l2, boot=bt_out, boot_in=bt_in),
          dict(kind=K.CKKS_LAYER_BLOCK, convs=m2_l3, boot=bt_out)]
    m3 = [dict(kind=K.CKKS_LAYER_BLOCK, convs=m3_l1, boot=b1),
          dict(kind=K.CKKS_LAYER_BLOCK, convs=m3_l2, boot=b1, inputs=[[1], [0]], n_in=2),
          dict(kind=K.CKKS_LAYER_BLOCK, convs=m3_l3, boot=b1)]
    m4 = [dict(kind=K.CKKS_LAYER_BLOCK, convs=m4_l1, boot=bt_in),
          dict(kind=K.CKKS_LAYER_DOWNSAMPLE, convs=m4_l2, boot=bt_out, boot_in=bt_in, inputs=[[0], [1]], n_in=2),
          dict(kind=K.CKKS_LAYER_BLOCK, convs=m4_l3, boot=bt_out)]

    def make_input(seed):
        x = WL.image(seed, C, w0)
        ct = K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, x, w, 1, delta[1]), seed)
        return K.ckks_ct_export_rns(ctx, ct)

    def eager_m1(limbs, keys=keys):
        x = K.ckks_ct_import_rns(ctx, limbs, 1, delta[1])
        ys = [K.ckks_level_down(ctx, K.ckks_block(ctx, keys, x, m1_l1[j][0], b1), 1) for j in range(2)]
        return K.ckks_ct_export_rns(ctx, K.ckks_block_multi(ctx, keys, ys, m1_l2[0], b1))

    def eager_m2(limbs):
        x = K.ckks_ct_import_rns(ctx, limbs, 1, delta[1])
        re, im = K.ckks_bootstrap(ctx, keys, bt_in, K.ckks_conv2d_cins(ctx, keys, x, m2_l1[0][0]))
        y = K.ckks_downsample_layer(ctx, keys, [re], [im], bt_in, m2_l2[0], bt_out)
        y = K.ckks_level_down(ctx, y, 1)
        return K.ckks_ct_export_rns(ctx, K.ckks_block(ctx, keys, y, m2_l3[0][0], bt_out))

    def eager_m3(limbs):
        x = K.ckks_ct_import_rns(ctx, limbs, 1, delta[1])
        ys = [K.ckks_level_down(ctx, K.ckks_block(ctx, keys, x, m3_l1[j][0], b1), 1) for j in range(2)]
        zs = [K.ckks_level_down(ctx, K.ckks_block(ctx, keys, ys[1 - j], m3_l2[j][0], b1), 1) for j in range(2)]
        return K.ckks_ct_export_rns(ctx, K.ckks_block_multi(ctx, keys, zs, m3_l3[0], b1))

    def eager_m4(limbs):
        x = K.ckks_ct_import_rns(ctx, limbs, 1, delta[1])
        ds = []
        for j in range(2):
            re, im = K.ckks_bootstrap(ctx, keys, bt_in, K.ckks_conv2d_cins(ctx, keys, x, m4_l1[j][0]))
            d = K.ckks_downsample_layer(ctx, keys, [re], [im], bt_in, m4_l2[j], bt_out)
            ds.append(K.ckks_level_down(ctx, d, 1))
        return K.ckks_ct_export_rns(ctx, K.ckks_block_multi(ctx, keys, ds, m4_l3[0], bt_out))

    # model M5: the second layer of M1 alone (two input ciphertexts: larger requests than M1's)
    m5 = [dict(kind=K.CKKS_LAYER_BLOCK, convs=m1_l2, boot=b1)]

    def eager_m5(limbs2, keys=keys):
        xs = [K.ckks_ct_import_rns(ctx, limbs2[t], 1, delta[1]) for t in range(2)]
        return K.ckks_ct_export_rns(ctx, K.ckks_block_multi(ctx, keys, xs, m1_l2[0], b1))

    def model_rotations(layers):
        r = set()
        for L in layers:
            for row in L["convs"]:
                for p in row:
                    r |= set(K.ckks_ptset_rotations(p))
            for b in (L["boot"], L.get("boot_in")):
                if b is not None:
                    r |= set(K.ckks_boot_rotations(b))
        return r

    return dict(K=K, ctx=ctx, keys=keys, rots=rots, m1=m1, m2=m2, m3=m3, m4=m4, m5=m5, make_input=make_input,
                eager_m1=eager_m1, eager_m2=eager_m2, eager_m3=eager_m3, eager_m4=eager_m4, eager_m5=eager_m5,
                model_rotations=model_rotations, delta=delta)


def _server(env, slots):
    K = env["K"]
    srv = K.ckks_server_create(env["ctx"], env["keys"], slots, 0)
    a = K.ckks_server_add_model_layers(srv, env["m1"])
    b = K.ckks_server_add_model_layers(srv, env["m2"])
    K.ckks_server_start(srv)
    return srv, a, b


def test_layer_models_match_eager_calls_alone_and_in_a_mix(env):
    K, ctx = env["K"], env["ctx"]
    n = ctx.n
    ins = {s: env["make_input"](s) for s in (5, 6, 7, 8)}
    want = {5: env["eager_m1"](ins[5]), 6: env["eager_m2"](ins[6]), 7: env["eager_m1"](ins[7]),
            8: env["eager_m2"](ins[8])}
    srv, a, b = _server(env, 4)
    try:
        assert K.ckks_server_model_shape(srv, a) == (1, 1) and K.ckks_server_model_shape(srv, b) == (1, 1)
        model = {5: a, 6: b, 7: a, 8: b}
        # alone: one request at a time
        for s in (5, 6):
            rid = K.ckks_server_submit(srv, model[s], ins[s], 1, env["delta"][1])
            assert K.ckks_server_wait(srv, rid, 120.0) == K.CKKS_REQ_DONE
            out, lev, _ = K.ckks_server_result(srv, rid, n)
            assert (out == want[s]).all(), s
        # in a mix: all four in flight together, several rounds
        for _ in range(2):
            rids = {s: K.ckks_server_submit(srv, model[s], ins[s], 1, env["delta"][1]) for s in (5, 6, 7, 8)}
            for s, rid in rids.items():
                assert K.ckks_server_wait(srv, rid, 120.0) == K.CKKS_REQ_DONE
                out, _, _ = K.ckks_server_result(srv, rid, n)
                assert (out == want[s]).all(), s
    finally:
        srv.close()


def test_layer_model_checks(env):
    K = env["K"]
    srv = K.ckks_server_create(env["ctx"], env["keys"], 1, 0)
    try:
        m2 = env["m2"]
        with pytest.raises(K.CkksError):        # a downsampling layer cannot come first
            K.ckks_server_add_model_layers(srv, m2[1:])
        with pytest.raises(K.CkksError):        # input count differs from the previous outputs
            K.ckks_server_add_model_layers(srv, [env["m1"][0], m2[2]])
        bad = dict(m2[1])
        bad["boot_in"] = None
        with pytest.raises(K.CkksError):        # a downsampling layer needs bt_in
            K.ckks_server_add_model_layers(srv, [m2[0], bad, m2[2]])
        bad = dict(env["m3"][1])
        bad["inputs"] = [[2], [0]]
        with pytest.raises(K.CkksError):        # an input index out of range
            K.ckks_server_add_model_layers(srv, [env["m3"][0], bad, env["m3"][2]])
    finally:
        srv.close()


def test_outputs_reading_chosen_inputs(env):
    """block and downsampling layers whose outputs each read one chosen input ciphertext (the
    ResNet-18 pooling and stage-entry pattern), against the same layers called eagerly"""
    K, ctx = env["K"], env["ctx"]
    n = ctx.n
    ins = {s: env["make_input"](s) for s in (11, 12)}
    want = {11: env["eager_m3"](ins[11]), 12: env["eager_m4"](ins[12])}
    srv = K.ckks_server_create(ctx, env["keys"], 2, 0)
    try:
        a = K.ckks_server_add_model_layers(srv, env["m3"])
        b = K.ckks_server_add_model_layers(srv, env["m4"])
        K.ckks_server_start(srv)
        rids = {11: K.ckks_server_submit(srv, a, ins[11], 1, env["delta"][1]),
                12: K.ckks_server_submit(srv, b, ins[12], 1, env["delta"][1])}
        for s, rid in rids.items():
            assert K.ckks_server_wait(srv, rid, 120.0) == K.CKKS_REQ_DONE
            out, _, _ = K.ckks_server_result(srv, rid, n)
            assert (out == want[s]).all(), s
    finally:
        srv.close()


def test_failed_model_between_models_of_different_request_sizes(env):
    """one server, three models added in turn: M1 (one input ciphertext); M2, refused while it
    is recorded because the server's keys lack one of its rotations (CKKS_ENOKEY from its eager
    run, after its staging buffers were made); M5 (two input ciphertexts, larger requests than
    M1's).  Each model keeps its own staging buffers, so M1's recorded graphs stay valid after
    the larger model is added, and the refused model leaves no trace: requests of M1 and M5,
    alone and mixed, equal the same layers called eagerly with the same keys"""
    K, ctx = env["K"], env["ctx"]
    n = ctx.n
    keep = env["model_rotations"](env["m1"]) | env["model_rotations"](env["m5"])
    only_m2 = sorted(env["model_rotations"](env["m2"]) - keep)
    if not only_m2:
        pytest.skip("every rotation of M2 is also one of M1's or M5's")
    short = K.ckks_keygen(ctx, sorted(set(env["rots"]) - {only_m2[0]}), True)
    x1 = env["make_input"](21)
    x5 = np.stack([env["make_input"](22), env["make_input"](23)])
    want1 = env["eager_m1"](x1, short)
    want5 = env["eager_m5"](x5, short)
    srv = K.ckks_server_create(ctx, short, 2, 0)
    try:
        a = K.ckks_server_add_model_layers(srv, env["m1"])
        with pytest.raises(K.CkksError) as ei:
            K.ckks_server_add_model_layers(srv, env["m2"])
        assert ei.value.code == K.CKKS_ENOKEY
        b = K.ckks_server_add_model_layers(srv, env["m5"])
        assert b == a + 1
        assert K.ckks_server_model_shape(srv, a) == (1, 1) and K.ckks_server_model_shape(srv, b) == (2, 1)
        K.ckks_server_start(srv)
        for _ in range(2):
            rids = [(K.ckks_server_submit(srv, a, x1, 1, env["delta"][1]), want1),
                    (K.ckks_server_submit(srv, b, x5, 1, env["delta"][1]), want5),
                    (K.ckks_server_submit(srv, a, x1, 1, env["delta"][1]), want1)]
            for rid, want in rids:
                assert K.ckks_server_wait(srv, rid, 120.0) == K.CKKS_REQ_DONE
                out, _, _ = K.ckks_server_result(srv, rid, n)
                assert (out == want).all()
    finally:
        srv.close()
