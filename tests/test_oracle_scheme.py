"""Pins of the oracle's scheme layer: what decrypts must equal the plaintext-side
computation the paper states (rotation = slot roll, conj, products, BSGS = matrix
product, conv = FP64 conv2d, EvalMod = sine), plus the Table 1 operation counts."""
import json
import math
import os

import numpy as np
import pytest

from oracle import boot as BT
from oracle import encoding as E
from oracle import params as PP
from oracle.scheme import Oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(11)


@pytest.fixture(scope="module")
def small():
    P = PP.Params(9, 6, 3, 60, 40, 60, h=32)
    o = Oracle(P, 42)
    o.gen_relin_key()
    o.gen_conj_key()
    o.gen_rotation_keys([1, 3, 7, 100])
    return o


def slots(o, ct):
    return o.decode_slots(o.decrypt(ct))


def cvec(n):
    return rng.normal(size=n) + 1j * rng.normal(size=n)


def test_encrypt_decrypt(small):
    o = small
    m = o.P.n // 2
    z = cvec(m)
    for lev in (o.P.L, 2, 0):
        pt = o.encode_pt(z, lev, o.P.delta[lev])
        assert np.abs(slots(o, o.encrypt(pt, 1)) - z).max() < 1e-6
        assert np.abs(slots(o, o.encrypt_sk(pt, 2)) - z).max() < 1e-6
        # decode(encode) without encryption is exact to the rounding of the encoding
        assert np.abs(o.decode_slots(pt) - z).max() < 1e-9


def test_rotation_conjugation_product(small):
    o = small
    m = o.P.n // 2
    z = cvec(m)
    L = o.P.L
    ct = o.encrypt(o.encode_pt(z, L, o.P.delta[L]), 3)
    outs = o.rotate_hoisted(ct, [0, 1, 3, 7, 100])
    for r, c in zip([0, 1, 3, 7, 100], outs):
        assert np.abs(slots(o, c) - np.roll(z, -r)).max() < 1e-6       # HRot: slot j <- j + r
    assert np.abs(slots(o, o.conjugate(ct)) - np.conj(z)).max() < 1e-6
    sq = o.rescale(o.mul_relin(ct, ct))
    assert sq.scale == o.P.delta[L - 1]                                 # canonical ladder
    assert np.abs(slots(o, sq) - z * z).max() < 1e-5
    im = o.imult(ct)
    assert np.abs(slots(o, im) - 1j * z).max() < 1e-6
    down = o.level_down(ct, 1)
    assert down.level == 1 and abs(down.scale - o.P.delta[1]) < 1e-9 * down.scale
    assert np.abs(slots(o, down) - z).max() < 1e-5
    c = o.add_const(ct, 0.75)
    assert np.abs(slots(o, c) - (z + 0.75)).max() < 1e-6


def test_theorem1_under_encryption(small):
    """Theorem 1 / Eq. 5 homomorphically: the folded slices P_l m_i in slot encoding, taken
    through S_{l<-1} as the StoC1 BSGS levels under encryption, decrypt to the direct
    real-CinS encoding of the slices (the partial DFT of slot encoding is CinS)"""
    o = small
    P = o.P
    n, m = P.n, P.n // 2
    ell = 8
    C = m // ell
    sl = 0.5 * rng.normal(size=(C, 2 * ell))
    z = np.kron(np.eye(C), E.P_matrix(ell)) @ np.concatenate([E.fold(v) for v in sl])
    assert np.abs(z - E.real_cins_slots(sl)).max() > 0.1              # the map is not trivial
    lev = P.L
    ct = o.encrypt(o.encode_pt(z, lev, P.delta[lev]), 8)
    for D, strides in E.stoc1_groups(n, ell, 2):
        a0, step, count = E.ap_of_group(strides, m)
        plan = o.make_plan(D, a0, step, count, lev, float(P.q[lev]))
        o.gen_rotation_keys(plan.rotations(m))
        ct = o.rescale(o.bsgs(ct, plan))
        lev -= 1
    assert ct.level == P.L - 2
    assert np.abs(slots(o, ct) - E.real_cins_slots(sl)).max() < 1e-5


def test_mod_raise_overflow_is_small_multiple_of_q0(small):
    o = small
    m = o.P.n // 2
    ct = o.encrypt(o.encode_pt(cvec(m) * 0.1, 0, 2.0 ** 30), 4)
    t0 = o.centred_coeffs(o.decrypt(ct))
    raised = o.mod_raise(ct)
    t = o.centred_coeffs(o.decrypt(raised))
    I = (t - t0) / float(o.P.q[0])
    assert np.allclose(I, np.round(I))
    assert np.abs(I).max() <= (o.P.h + 1) / 2


def test_bsgs_equals_matrix_product(small):
    """Eq. 3 with the BSGS split (Sec. 2.5) on a sparse matrix with AP diagonals"""
    o = small
    m = o.P.n // 2
    L = o.P.L
    a0, step, count = m - 6, 3, 5
    diags = {(a0 + step * i) % m: cvec(m) * 0.3 for i in range(count)}
    o.gen_rotation_keys([step * b for b in range(1, 4)] + [(a0 + step * 2 * g) % m for g in range(3)]
                        + [(a0 + step * 4 * g) % m for g in range(2)])
    z = cvec(m)
    ct = o.encrypt(o.encode_pt(z, L, o.P.delta[L]), 5)
    want = E.diag_apply(diags, z)
    for B in (1, 2, 4):
        o.gen_rotation_keys([(a0 + step * B * g) % m for g in range(-(-count // B))])
        plan = o.make_plan(diags, a0, step, count, L, float(o.P.q[L]), B)
        out = o.rescale(o.bsgs(ct, plan))
        assert np.abs(slots(o, out) - want).max() < 1e-5


def test_cfg1_conv_matches_fp64_and_table1():
    """config-1 shape: fused CinS conv == FP64 conv2d; op counts = Table 1 (C PMult,
    2 sqrt(C) - 2 HRot, one rescale)"""
    gold = json.load(open(os.path.join(GOLD, "table1_op_counts.json")))
    assert gold["conv2d"]["pmult"] == "C" and gold["conv2d"]["hrot"] == "2*sqrt(C)-2"
    P = PP.cfg1_params()
    o = Oracle(P, 1)
    x = rng.random((1, 16, 16))
    W = rng.uniform(-1, 1, (1, 1, 3, 3))
    w = E.pad_width(16, 3)
    C = P.n // (w * w)
    z = E.cins_input_slots(x, w, P.n)
    for lev in (P.L, 1):
        ct = o.encrypt(o.encode_pt(z, lev, P.delta[lev]), 3)
        plan = o.conv_plan(W, 1, 1, 3, w, lev, (P.delta[lev - 1] * float(P.q[lev])) / ct.scale)
        o.gen_rotation_keys(plan.rotations(P.n // 2))
        o.ops = {k: 0 for k in o.ops}
        out = o.conv2d_cins(ct, plan)
        assert o.ops["pmult"] == C and o.ops["hrot"] == 2 * math.isqrt(C) - 2
        assert out.level == lev - 1 and o.ops["rescale"] == 1
        got = E.conv_output_from_coeffs(o.decode_coeffs(o.decrypt(out)), C, w * w, 1, w, 16)
        assert np.abs(got - E.conv2d_same(x, W)).max() < 1e-6


def test_full_channel_conv_op_counts():
    """C = C_in = C_out = 16 channels per ciphertext: 16 PMult and 6 HRot (Table 1)"""
    P = PP.Params(10, 3, 1, 60, 42, 60)
    o = Oracle(P, 2)
    w0, w = 4, 8
    C = P.n // (w * w)
    x = rng.random((C, w0, w0))
    W = rng.normal(0, 0.1, (C, C, 3, 3))
    ct = o.encrypt(o.encode_pt(E.cins_input_slots(x, w, P.n), 1, P.delta[1]), 1)
    plan = o.conv_plan(W, C, C, 3, w, 1, (P.delta[0] * float(P.q[1])) / ct.scale)
    o.gen_rotation_keys(plan.rotations(P.n // 2))
    o.ops = {k: 0 for k in o.ops}
    out = o.conv2d_cins(ct, plan)
    assert o.ops["pmult"] == 16 and o.ops["hrot"] == 6
    got = E.conv_output_from_coeffs(o.decode_coeffs(o.decrypt(out)), C, w * w, C, w, w0)
    assert np.abs(got - E.conv2d_same(x, W)).max() < 1e-6


def test_chebyshev_and_evalmod(small):
    o = small
    P = o.P
    m = P.n // 2
    y = rng.uniform(-1, 1, m)
    L = P.L
    ct = o.encrypt(o.encode_pt(y, L, P.delta[L]), 6)
    coeffs = np.polynomial.chebyshev.chebinterpolate(lambda t: np.sin(3 * t) + 0.5 * t * t, 5)
    out = o.cheb_eval(ct, list(coeffs))
    assert out.level == L - math.ceil(math.log2(5)) - 1
    assert np.abs(slots(o, out).real - np.polynomial.chebyshev.chebval(y, coeffs)).max() < 1e-5


def test_evalmod_function_is_the_scaled_sine():
    """EvalMod in FP64 with the bootstrapping configuration's own coefficients (Chebyshev
    interpolant of cos(2 pi (K_eff y - 1/4) / 2^r), then r double angles c <- 2 c^2 - 1)
    against sin(2 pi K_eff y) on the intervals where ModRaise puts t / (q0 K_eff): y = (k + u)
    / K_eff, |k| < K, |u| <= 2^-9 (a message ratio Delta0 / q0 = 2^-11 with |o| up to 4).
    Then the masks' factor q0 / (2 pi Delta0) returns o up to the sine's cubic term, whose
    closed form |o| (2 pi u)^2 / 6 bounds the error for |o| <= 1."""
    from tests.pairs import oracle_params
    P = oracle_params("cfg2_small")              # the config-2 chain at N = 2^10
    cfg = BT.BootConfig(Oracle(P, 5), 8, 4, 4)
    c = np.array(cfg.coeffs)
    assert len(c) == cfg.deg + 1 and cfg.r == 3 and abs(cfg.K_eff - cfg.K) < 1e-6
    u = np.linspace(-2.0 ** -9, 2.0 ** -9, 1025)
    ratio = cfg.delta0 / float(P.q[0])
    worst = worst_o = 0.0
    for k in range(-cfg.K + 1, cfg.K):
        y = (k + u) / cfg.K_eff
        v = np.polynomial.chebyshev.chebval(y, c)
        for _ in range(cfg.r):
            v = 2.0 * v * v - 1.0
        worst = max(worst, np.abs(v - np.sin(2.0 * np.pi * cfg.K_eff * y)).max())
        small_o = np.abs(u) <= ratio                      # |o| <= 1
        o_rec = v[small_o] / (2.0 * np.pi * ratio)        # masks: q0 / (2 pi Delta0)
        worst_o = max(worst_o, np.abs(o_rec - u[small_o] / ratio).max())
    assert worst < 1e-11, worst
    assert worst_o <= (2.0 * np.pi * ratio) ** 2 / 6.0 * 1.01 + 1e-12, worst_o
    assert worst_o < 2.0 ** -12 / 100


@pytest.mark.slow
def test_block_matches_fp64_conv():
    """Alg. 1 block (no activation) at N = 2^10 with the config-2 prime chain: decoded output
    is the masked conv output within 2^-12 (the accuracy bar of the GPU path)"""
    P = PP.Params(10, 24, 3, 60, 42, 60, h=192, n_p=7, boot_bits=48, n_boot=14)
    o = Oracle(P, 5)
    w0, w, f = 4, 8, 3
    n = P.n
    C = n // (w * w)
    cin = cout = 4
    x = rng.random((cin, w0, w0))
    W = rng.normal(0, 0.1, (cout, cin, f, f))
    ct = o.encrypt(o.encode_pt(E.cins_input_slots(x, w, n), 1, P.delta[1]), 3)
    cfg = BT.BootConfig(o, w, w0, cout)
    plan = o.conv_plan(W, cin, cout, f, w, 1, (cfg.delta0 * float(P.q[1])) / ct.scale)
    o.gen_rotation_keys(BT.block_rotations(o, plan, cfg))
    o.gen_conj_key()
    o.gen_relin_key()
    out = BT.block(o, ct, plan, cfg)
    assert out.level == cfg.l_out
    # the block one step at a time (how the CPU baseline times it) is the same ciphertext
    v = [ct]
    for _, step in BT.block_stages(o, plan, cfg):
        v = step(v)
    assert len(v) == 1 and (v[0].c0 == out.c0).all() and (v[0].c1 == out.c1).all()
    got = slots(o, out)
    ell = w * w // 2
    pix = np.stack([E.encode(got[i * ell:(i + 1) * ell], w * w) for i in range(C)])
    ref = np.zeros((C, w * w))
    conv = E.conv2d_same(x, W)
    for i in range(cout):
        ref[i] = E.flatten_padded(conv[i], w)
    assert np.abs(pix - ref).max() < 2.0 ** -12


def test_composite_relu_fit_and_eval():
    """the fitted stages meet their minimax bounds on a dense grid; the composite is odd in
    its sign part; decrypting the HActivation gives the FP64 polynomial ReLU"""
    from oracle import relu as R
    stages, info = R.composite_relu_stages()
    assert [i["deg"] for i in info] == [15, 15, 27]
    x = np.linspace(info[0]["eps"], 1, 20001)
    y = x.copy()
    for k, (s, inf) in enumerate(zip(stages, info)):
        y = np.polynomial.chebyshev.chebval(y, s)
        if k < len(stages) - 1:
            # the LP is solved on a grid: off-grid points may exceed its bound by a hair
            assert y.min() >= (1 - inf["tau"]) / (1 + inf["tau"]) - 1e-7 and y.max() <= 1 + 1e-7
    # g = (1 + sign)/2 ~ 1 on [eps, 1] within the last stage's tau / 2
    assert np.abs(y - 1).max() <= info[-1]["tau"] / 2 + 1e-7
    assert info[-1]["tau"] < 1e-5
    xs = np.linspace(-1, 1, 4001)
    relu = R.relu_poly_fp64(xs, stages)
    assert np.abs(relu - np.maximum(xs, 0)).max() <= info[0]["eps"]
    # encrypted evaluation at small N
    P = PP.Params(9, 20, 3, 60, 42, 60, h=32)
    o = Oracle(P, 8)
    o.gen_relin_key()
    m = P.n // 2
    v = np.random.default_rng(2).uniform(-1, 1, m)
    ct = o.encrypt(o.encode_pt(v, P.L, P.delta[P.L]), 1)
    out = R.relu_eval(o, ct, stages)
    assert out.level == P.L - 17
    got = slots(o, out).real
    assert np.abs(got - R.relu_poly_fp64(v, stages)).max() < 2.0 ** -12


def test_relu_across_segment_boundary():
    """on the two-segment chain (48-bit bootstrapping levels over 42-bit circuit levels) the
    composite ReLU, which runs across the boundary, still decodes to the FP64 polynomial"""
    from oracle import relu as R
    stages, _ = R.composite_relu_stages()
    P = PP.Params(9, 24, 3, 60, 42, 60, h=32, n_p=7, boot_bits=48, n_boot=14)
    o = Oracle(P, 43)
    o.gen_relin_key()
    v = np.random.default_rng(6).uniform(-1, 1, P.n // 2)
    out = R.relu_eval(o, o.encrypt(o.encode_pt(v, P.L, P.delta[P.L]), 1), stages)
    assert out.level == P.L - 18          # 17 levels + 1 for the boundary
    assert np.abs(slots(o, out).real - R.relu_poly_fp64(v, stages)).max() < 2.0 ** -12


def test_dwconv_one_pmult():
    """depthwise conv (Sec. 3.3.4, Table 1 row Dwconv2d: 1 PMult, 0 HRot, 1 level) decodes to
    FP64 depthwise conv2d at the real pixels"""
    P = PP.Params(10, 3, 1, 60, 42, 60)
    o = Oracle(P, 3)
    w0, w, f = 5, 8, 3
    C = P.n // (w * w)
    x = rng.random((C, w0, w0))
    K = rng.normal(0, 0.3, (C, f, f))
    ct = o.encrypt(o.encode_pt(E.cins_input_slots(x, w, P.n), 2, P.delta[2]), 1)
    pk = o.encode_pt(E.dwconv_kernel_slots(K, w, P.n), 2, P.delta[2])
    o.ops = {k: 0 for k in o.ops}
    out = o.dwconv_cins(ct, pk)
    assert o.ops["pmult"] == 1 and o.ops["hrot"] == 0 and out.level == 1
    z = slots(o, out)
    ell = w * w // 2
    pix = np.stack([E.encode(z[i * ell:(i + 1) * ell], w * w).reshape(w, w)[:w0, :w0] for i in range(C)])
    assert np.abs(pix - E.dwconv_same(x, K)).max() < 1e-6


def test_fc_fused_with_stoc():
    """FC fused with the whole StoC (Sec. 4.3, slot encoding = CinS with l = 1): V M equals the
    explicit special-DFT product; the homomorphic layer leaves M x in the coefficients; it takes
    log2(N/2 / n_in) replication rotations plus the BSGS rotations over n_in diagonals, 1 level"""
    P = PP.Params(10, 3, 1, 60, 42, 60)
    o = Oracle(P, 8)
    n, m = P.n, P.n // 2
    n_in, n_out = 16, 40
    M = rng.normal(0, 0.3, (n_out, n_in))
    F = E.fc_stoc_matrix(M, n)
    Mfull = np.zeros((m, n_in))
    Mfull[:n_out] = M
    assert np.abs(F - E.V_matrix(n) @ Mfull).max() < 1e-9
    x = np.zeros(m)
    x[:n_in] = rng.uniform(-1, 1, n_in)
    lev = 2
    ct = o.encrypt(o.encode_pt(x, lev, P.delta[lev]), 4)
    plan = o.fc_plan(M, lev, (P.delta[lev - 1] * float(P.q[lev])) / ct.scale)
    o.gen_rotation_keys(plan.rotations(m) + o.fc_replicate_steps(n_in))
    o.ops = {k: 0 for k in o.ops}
    out = o.fc_stoc(ct, plan, n_in)
    B = plan.B
    G = -(-n_in // B)
    assert o.ops["hrot"] == int(np.log2(m // n_in)) + (B - 1) + (G - 1)
    assert out.level == lev - 1
    y = o.decode_coeffs(o.decrypt(out))
    assert np.abs(y[:n_out] - M @ x[:n_in]).max() < 1e-6
    assert np.abs(y[n_out:]).max() < 1e-6


@pytest.mark.parametrize("a,b,basis", [(0.0, 4.0, "cheb"), (-3.0, 1.0, "power"), (-1.0, 1.0, "power")])
def test_eval_poly_intervals_and_bases(small, a, b, basis):
    """p on [a, b] in the Chebyshev basis of the interval (sum c_k T_k((2x - a - b) / (b - a))) or
    in the power basis (sum c_k x^k), decoded against numpy's evaluation of the same p"""
    o = small
    P = o.P
    m = P.n // 2
    x = rng.uniform(a, b, m)
    L = P.L
    ct = o.encrypt(o.encode_pt(x, L, P.delta[L]), 9)
    c = list(rng.normal(0, 0.3, 6))
    out = o.eval_poly(ct, c, a, b, basis)
    if basis == "cheb":
        want = np.polynomial.chebyshev.chebval((2 * x - a - b) / (b - a), c)
    else:
        want = np.polynomial.polynomial.polyval(x, c)
    extra = 0 if (a, b) == (-1.0, 1.0) else 1
    assert out.level == L - extra - math.ceil(math.log2(5)) - 1
    assert np.abs(slots(o, out).real - want).max() < 1e-4 * max(1.0, np.abs(want).max())
