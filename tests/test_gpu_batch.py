"""Lockstep batches (ckks_block_batched): B ciphertexts through one block with every kernel
launched once for the batch.  Each output must be the ciphertext the oracle's block gives for
its input (bit-exact), and the same as ckks_block on that input alone; the recorded graph of
the batch gives the eager batch's ciphertexts."""
import numpy as np
import pytest

import workloads as WL
from oracle import boot as BT
from oracle import encoding as E
from tests.pairs import assert_ct_equal, gpu_ctx, import_plan, import_pt, make_pair, oracle_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def setup_module(module):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_04356_gb300 import build
    build.build()


def _setup(name, seed, spec, B, oracle_keys=True):
    """oracle and library with the oracle's plans imported, B seeded inputs"""
    from oracle.scheme import Oracle
    P = oracle_params(name)
    w = E.pad_width(spec["w0"], spec["f"])
    W = WL.weights(seed, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    o0 = Oracle(P, seed)
    cfg = BT.BootConfig(o0, w, spec["w0"], spec["cout"])
    plan = o0.conv_plan(W, spec["cin"], spec["cout"], spec["f"], w, 1, (cfg.delta0 * float(P.q[1])) / P.delta[1])
    rots = BT.block_rotations(o0, plan, cfg)
    K, o, ctx, keys = make_pair(name, seed, rotations=rots if oracle_keys else [])
    if not oracle_keys:
        keys = K.ckks_keygen(ctx, rots, True)
    cfg = BT.BootConfig(o, w, spec["w0"], spec["cout"])
    bt = K.ckks_boot_create(ctx, w, spec["w0"], spec["cout"])
    for i, p in enumerate(cfg.ctos):
        K.ckks_boot_set_ctos(ctx, bt, i, import_plan(K, ctx, p))
    for i, p in enumerate(cfg.stoc):
        K.ckks_boot_set_stoc(ctx, bt, i, import_plan(K, ctx, p))
    K.ckks_boot_set_coeffs(ctx, bt, cfg.coeffs)
    K.ckks_boot_set_masks(ctx, bt, import_pt(K, ctx, cfg.pt_mask_re), import_pt(K, ctx, cfg.pt_mask_im))
    pts = [o.encode_pt(E.cins_input_slots(WL.image(seed + 10 * b, spec["cin"], spec["w0"]), w, P.n), 1, P.delta[1])
           for b in range(B)]
    gcts = [K.ckks_encrypt(ctx, keys, import_pt(K, ctx, pt), 3 + b) for b, pt in enumerate(pts)]
    return dict(K=K, o=o, ctx=ctx, keys=keys, cfg=cfg, plan=plan, bt=bt, pts=pts, gcts=gcts,
                gplan=import_plan(K, ctx, plan))


def test_batched_block_bitexact_against_the_oracle():
    """B = 4 inputs on the config-2 chain at N = 2^10 (4 channels of 4 x 4): every output of the
    lockstep batch equals the oracle's block of its input on every limb"""
    d = _setup("cfg2_small", 51, WL.CONV["cfg2_small"], 4)
    K, o, ctx, keys = d["K"], d["o"], d["ctx"], d["keys"]
    outs = K.ckks_block_batched(ctx, keys, d["gcts"], d["gplan"], d["bt"])
    for b, (pt, out) in enumerate(zip(d["pts"], outs)):
        want = BT.block(o, o.encrypt(pt, 3 + b), d["plan"], d["cfg"])
        assert_ct_equal(K, ctx, out, want, "batched block, input %d" % b)


def test_batched_block_graph_and_side_streams():
    """the batch recorded as one CUDA graph, replayed twice (also after a new input is written),
    and the batch run without side streams, give ckks_block's ciphertext for every input"""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        d = _setup("cfg2_small", 52, WL.CONV["cfg2_small"], 3, oracle_keys=False)
        K, ctx, keys = d["K"], d["ctx"], d["keys"]
        want = [K.ckks_ct_export_rns(ctx, K.ckks_block(ctx, keys, c, d["gplan"], d["bt"])) for c in d["gcts"]]
        outs = [K.ckks_ct_create(ctx) for _ in d["gcts"]]
        g = K.ckks_block_batched_graph_create(ctx, keys, d["gcts"], d["gplan"], d["bt"], outs)
        for _ in range(2):
            K.ckks_graph_launch(g)
            K.ckks_sync(ctx)
            for w_, out in zip(want, outs):
                assert (K.ckks_ct_export_rns(ctx, out) == w_).all()
        K.ckks_ct_copy_into(ctx, d["gcts"][0], d["gcts"][2])           # a new input in the same handle
        K.ckks_graph_launch(g)
        K.ckks_sync(ctx)
        assert (K.ckks_ct_export_rns(ctx, outs[2]) == want[0]).all()
        K.ckks_ctx_set_side_streams(ctx, 0)
        eager = K.ckks_block_batched(ctx, keys, d["gcts"][:2], d["gplan"], d["bt"])
        K.ckks_ctx_set_side_streams(ctx, 1)
        for w_, out in zip(want, eager):
            assert (K.ckks_ct_export_rns(ctx, out) == w_).all()


def test_batched_block_with_stored_babies():
    """64 slices per ciphertext (w = 4 at N = 2^10, 16 channels): the conv's BSGS has 8 giant
    steps, so the batch takes the stored-baby path (hoisted rotations kept, then the inner sums
    of up to 8 giant steps per pass); every output equals ckks_block on its input alone, and
    the first also the oracle's block"""
    spec = dict(cin=16, cout=16, w0=2, f=3, weight="gauss")
    d = _setup("cfg2_small", 53, spec, 2)
    K, o, ctx, keys = d["K"], d["o"], d["ctx"], d["keys"]
    assert d["plan"].G > 4
    outs = K.ckks_block_batched(ctx, keys, d["gcts"], d["gplan"], d["bt"])
    for c, out in zip(d["gcts"], outs):
        one = K.ckks_block(ctx, keys, c, d["gplan"], d["bt"])
        assert (K.ckks_ct_export_rns(ctx, out) == K.ckks_ct_export_rns(ctx, one)).all()
    want = BT.block(o, o.encrypt(d["pts"][0], 3), d["plan"], d["cfg"])
    assert_ct_equal(K, ctx, outs[0], want, "batched block, stored babies")


def test_batched_block_full_size():
    """N = 2^16, config 2, B = 2: the lockstep batch gives ckks_block's ciphertext for each input
    (ckks_block itself is bit-exact against the oracle at this size, test_gpu_parity), and the
    outputs decode within 2^-12 of FP64 conv2d"""
    from paper_2312_04356_gb300 import ckks as K
    spec = WL.CONV["cfg2"]
    w = E.pad_width(spec["w0"], spec["f"])
    ctx = gpu_ctx("cfg2", 54)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    bt = K.ckks_boot_create(ctx, w, spec["w0"], spec["cout"])
    W = WL.weights(54, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    conv = K.ckks_ptset_conv_fused(ctx, W, spec["cin"], spec["cout"], spec["f"], w, 1,
                                   (2.0 ** 49 * q[1]) / delta[1])
    keys = K.ckks_keygen(ctx, sorted(set(K.ckks_ptset_rotations(conv)) | set(K.ckks_boot_rotations(bt))), True)
    xs = [WL.image(54 + b, spec["cin"], spec["w0"]) for b in range(2)]
    cts = [K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, x, w, 1, delta[1]), 7 + b) for b, x in enumerate(xs)]
    outs = K.ckks_block_batched(ctx, keys, cts, conv, bt)
    for x, c, out in zip(xs, cts, outs):
        one = K.ckks_block(ctx, keys, c, conv, bt)
        assert (K.ckks_ct_export_rns(ctx, out) == K.ckks_ct_export_rns(ctx, one)).all()
        got = K.ckks_decode_image(ctx, K.ckks_decrypt(ctx, keys, out), spec["cout"], spec["w0"], w)
        assert np.abs(got - E.conv2d_same(x, W)[: spec["cout"]]).max() < 2.0 ** -12


def test_batched_block_arguments():
    d = _setup("cfg2_small", 55, WL.CONV["cfg2_small"], 2, oracle_keys=False)
    K, ctx, keys = d["K"], d["ctx"], d["keys"]
    with pytest.raises(K.CkksError):                                    # output aliases an input
        K.ckks_block_batched(ctx, keys, d["gcts"], d["gplan"], d["bt"], outs=[d["gcts"][1], K.ckks_ct_create(ctx)])
    low = K.ckks_rescale(ctx, K.ckks_mul_int(ctx, d["gcts"][1], 1))
    with pytest.raises(K.CkksError):                                    # inputs at different levels
        K.ckks_block_batched(ctx, keys, [d["gcts"][0], low], d["gplan"], d["bt"])


def test_batched_downsample_layer_equals_one_at_a_time():
    """Alg. 2 for B = 2 inputs (each two EvalMod output pairs of the config-2 chain at N = 2^10)
    as one lockstep batch: each output equals ckks_downsample_layer on that input alone"""
    from paper_2312_04356_gb300 import ckks as K
    spec = WL.CONV["cfg2_small"]
    w0, w, C = spec["w0"], E.pad_width(spec["w0"], spec["f"]), 16
    ctx = gpu_ctx("cfg2_small", 56)
    q, p, psi, delta = K.ckks_ctx_info(ctx)
    bt = K.ckks_boot_create(ctx, w, w0, spec["cout"])
    bt_in = K.ckks_boot_create(ctx, w, w0, C, stride=2)
    bt_out = K.ckks_boot_create(ctx, w // 2, w0 // 2, 4 * C)
    W = WL.weights(56, spec["cout"], spec["cin"], spec["f"], spec["weight"])
    conv = K.ckks_ptset_conv_fused(ctx, W, spec["cin"], spec["cout"], spec["f"], w, 1, (2.0 ** 49 * q[1]) / delta[1])
    W2 = WL.weights(57, 4 * C, 2 * C, 3, "normal")
    convs = [K.ckks_ptset_conv_fused_s2(ctx, W2, 2 * C, 4 * C, 3, w, t, 1, (2.0 ** 49 * q[1]) / delta[1])
             for t in range(2)]
    rots = set(K.ckks_ptset_rotations(conv))
    for o in (bt, bt_in, bt_out):
        rots |= set(K.ckks_boot_rotations(o))
    for o in convs:
        rots |= set(K.ckks_ptset_rotations(o))
    keys = K.ckks_keygen(ctx, sorted(rots), True)
    res, ims = [], []
    for b in range(2):
        rb, ib = [], []
        for t in range(2):
            x = WL.image(60 + 2 * b + t, spec["cin"], w0)
            ct = K.ckks_encrypt(ctx, keys, K.ckks_encode_image(ctx, x, w, 1, delta[1]), 60 + 2 * b + t)
            r_, i_ = K.ckks_bootstrap(ctx, keys, bt, K.ckks_conv2d_cins(ctx, keys, ct, conv))
            rb.append(r_)
            ib.append(i_)
        res.append(rb)
        ims.append(ib)
    outs = K.ckks_downsample_layer_batched(ctx, keys, res, ims, bt_in, convs, bt_out)
    for b in range(2):
        one = K.ckks_downsample_layer(ctx, keys, res[b], ims[b], bt_in, convs, bt_out)
        assert (K.ckks_ct_export_rns(ctx, outs[b]) == K.ckks_ct_export_rns(ctx, one)).all()


def test_batched_bootstrap_and_activation_equal_one_at_a_time():
    """ckks_bootstrap_batched, ckks_eval_poly_batched (on [0, 2]) and ckks_eval_relu_batched (the
    fitted composite (15, 15, 27)) for B = 3 inputs give each input's single-ciphertext result"""
    from oracle import relu as R
    d = _setup("cfg2_small", 58, WL.CONV["cfg2_small"], 3, oracle_keys=False)
    K, ctx, keys = d["K"], d["ctx"], d["keys"]
    x0s = [K.ckks_conv2d_cins(ctx, keys, c, d["gplan"]) for c in d["gcts"]]
    res, ims = K.ckks_bootstrap_batched(ctx, keys, d["bt"], x0s)
    for x0, r, i in zip(x0s, res, ims):
        r1, i1 = K.ckks_bootstrap(ctx, keys, d["bt"], x0)
        assert (K.ckks_ct_export_rns(ctx, r) == K.ckks_ct_export_rns(ctx, r1)).all()
        assert (K.ckks_ct_export_rns(ctx, i) == K.ckks_ct_export_rns(ctx, i1)).all()
    P = d["o"].P
    rng = np.random.default_rng(58)
    ins = [K.ckks_encrypt(ctx, keys, K.ckks_encode(ctx, rng.uniform(-1, 1, P.n // 2), P.L, P.delta[P.L]), 20 + b)
           for b in range(3)]
    c = list(rng.normal(0, 0.3, 8))
    polys = K.ckks_eval_poly_batched(ctx, keys, ins, c, K.CKKS_BASIS_CHEB, 0.0, 2.0)
    stages, _ = R.composite_relu_stages()
    relus = K.ckks_eval_relu_batched(ctx, keys, ins, stages)
    for x, po, re_ in zip(ins, polys, relus):
        p1 = K.ckks_eval_poly(ctx, keys, x, c, K.CKKS_BASIS_CHEB, 0.0, 2.0)
        assert (K.ckks_ct_export_rns(ctx, po) == K.ckks_ct_export_rns(ctx, p1)).all()
        q1 = K.ckks_eval_relu(ctx, keys, x, stages)
        assert (K.ckks_ct_export_rns(ctx, re_) == K.ckks_ct_export_rns(ctx, q1)).all()
