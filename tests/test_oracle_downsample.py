"""Oracle pins of the decomposed downsampling conv2d (Alg. 2, calG_l of Appendix B)."""
import numpy as np
import pytest

from oracle import boot as BT
from oracle import encoding as E
from oracle import params as PP
from oracle.scheme import Oracle

rng = np.random.default_rng(23)


def _perm_matrix(src):
    m = len(src)
    M = np.zeros((m, m))
    M[np.arange(m), src] = 1.0
    return M


@pytest.mark.parametrize("w", [8, 16])
def test_decomposition_is_the_polyphase_permutation(w):
    """Alg. 2's decomposition (calG_l with the rotations r and the shifts j l/4) equals the slot
    permutation derived from the layouts alone; every slot is moved exactly once; the offsets
    form the arithmetic progression the BSGS plan uses"""
    n = 4 * w * w
    m = n // 2
    D = E.decompose_diag(w, n)
    src = E.decompose_source(w, n)
    assert (src >= 0).all() and len(set(src.tolist())) == m
    assert np.array_equal(E.diag_to_dense(D, m), _perm_matrix(src))
    a0, step, count = E.decompose_ap(w, n)
    assert set(D) == {(a0 + step * i) % m for i in range(count)}


def test_literal_G_bound_is_not_a_permutation():
    """the appendix's bound i <= w/2 read literally adds block (w/2, w): that block writes the
    slots of the j = 1 term, so the composed map is no longer a permutation (reading: i < w/2)"""
    w = 8
    n = 4 * w * w
    m = n // 2
    ell, b = w * w // 2, w // 4
    G = E.G_matrix(w)
    G[(w // 2) * b:(w // 2 + 1) * b, w * b:(w + 1) * b] = np.eye(b)
    Gd = E.blockdiag_to_diag(G, m)
    r = [0, ell // 2, w // 4, ell // 2 + w // 4]
    D = {}
    for j in range(4):
        t = E.diag_mul(E.rotation_diag(-j * (ell // 4), m), E.diag_mul(Gd, E.rotation_diag(r[j], m), m), m)
        for o, v in t.items():
            D[o] = D[o] + v if o in D else v
    M = E.diag_to_dense(D, m)
    assert np.abs(M).sum(axis=1).max() > 1.0


def test_decomposition_moves_polyphase_pixels():
    """on the slot layout of the activation output (slot i l + rev_l(k) = x_k + i x_{k+l}), the
    decomposition gives the same layout of the polyphase images x[p::2, q::2]"""
    w, C = 8, 4
    n = C * w * w
    ell = w * w // 2
    x = rng.random((C, w, w))

    def layout(img, width):
        l_ = width * width // 2
        rev = E.bitrev_indices(l_)
        z = np.zeros(img.shape[0] * l_, dtype=np.complex128)
        for i in range(img.shape[0]):
            f = img[i].reshape(-1)
            z[i * l_ + rev] = f[:l_] + 1j * f[l_:]
        return z

    z = layout(x, w)
    got = E.diag_apply(E.decompose_diag(w, n), z)
    assert np.abs(got - layout(E.decompose_images(x), w // 2)).max() < 1e-12
    assert ell == 4 * (ell // 4)


def _conv_stride2_loops(x, W):
    cin, h, _ = x.shape
    cout, _, f, _ = W.shape
    c = f // 2
    out = np.zeros((cout, h // 2, h // 2))
    for o in range(cout):
        for y in range(h // 2):
            for xx in range(h // 2):
                s = 0.0
                for i in range(cin):
                    for a in range(f):
                        for b in range(f):
                            r, col = 2 * y + a - c, 2 * xx + b - c
                            if 0 <= r < h and 0 <= col < h:
                                s += W[o, i, a, b] * x[i, r, col]
                out[o, y, xx] = s
    return out


@pytest.mark.parametrize("f", [1, 3, 5])
def test_decomposed_kernels_give_the_stride2_conv(f):
    """sum over the two input ciphertexts of unit-stride convs of the polyphase images with
    the decomposed kernels == stride-2 conv2d (brute force, zero padding f//2)"""
    C, h = 3, 8
    x = rng.random((2 * C, h, h))
    W = rng.normal(size=(5, 2 * C, f, f))
    ref = _conv_stride2_loops(x, W)
    assert np.abs(E.conv2d_stride2(x, W) - ref).max() < 1e-12
    pp = E.decompose_images(x)
    acc = 0
    for t in range(2):
        acc = acc + E.conv2d_same(pp[4 * C * t:4 * C * (t + 1)], E.decompose_kernels(W, C, t))
    assert np.abs(acc - ref).max() < 1e-12


def _dwconv_stride2_loops(x, Kd):
    c_, h, _ = x.shape
    f = Kd.shape[1]
    c = f // 2
    out = np.zeros((c_, h // 2, h // 2))
    for i in range(c_):
        for y in range(h // 2):
            for xx in range(h // 2):
                for a in range(f):
                    for b in range(f):
                        r, col = 2 * y + a - c, 2 * xx + b - c
                        if 0 <= r < h and 0 <= col < h:
                            out[i, y, xx] += Kd[i, a, b] * x[i, r, col]
    return out


def _avgpool_stride2(x, f):
    """mean over the f x f windows at stride 2 of the zero-padded image (padding counted)"""
    c = f // 2
    h = x.shape[1]
    xp = np.pad(x, ((0, 0), (c, c), (c, c)))
    s = sum(xp[:, a:a + h:2, b:b + h:2] for a in range(f) for b in range(f))
    return s / (f * f)


@pytest.mark.parametrize("f", [3, 5])
def test_downsampling_dwconv_and_avgpool_through_the_decomposition(f):
    """Sec. 3.3.4: a downsampling depthwise conv is the stride-2 conv whose weights are
    diagonal (output channel i reads input channel i); through the decomposed kernels of the
    polyphase images it gives the strided depthwise conv (brute force), and with equal
    kernels 1/f^2 the stride-2 average pooling (window sums of the padded image)"""
    C, h = 3, 8
    x = rng.random((4 * C, h, h))
    Kd = rng.normal(size=(4 * C, f, f))
    W = np.zeros((4 * C, 4 * C, f, f))
    W[np.arange(4 * C), np.arange(4 * C)] = Kd
    pp = E.decompose_images(x)

    def through_decomposition(W):
        return sum(E.conv2d_same(pp[4 * C * t:4 * C * (t + 1)], E.decompose_kernels(W, C, t)) for t in range(4))

    assert np.abs(through_decomposition(W) - _dwconv_stride2_loops(x, Kd)).max() < 1e-12
    Wa = np.zeros_like(W)
    Wa[np.arange(4 * C), np.arange(4 * C)] = 1.0 / (f * f)
    assert np.abs(through_decomposition(Wa) - _avgpool_stride2(x, f)).max() < 1e-12
    # the decomposed kernels of input ciphertext t touch only output channels tC .. tC + C - 1
    for t in range(4):
        Wt = E.decompose_kernels(W, C, t)
        rows = np.flatnonzero(np.abs(Wt).reshape(4 * C, -1).sum(axis=1))
        assert set(rows.tolist()) <= set(range(t * C, (t + 1) * C))


def _tail_inputs(o, cfg, x, nonce):
    """Re / Im ciphertexts as the bootstrap hands them to the tail: slot i l + u holds pixel
    rev_l(u) (Re) or rev_l(u) + l (Im) of channel i, divided by the mask value; pixels outside
    the image carry garbage that the masks must remove"""
    P = o.P
    w, ell = cfg.w, cfg.ell
    val = float(P.q[0]) / (2.0 * np.pi * cfg.delta0)
    rev = E.bitrev_indices(ell)
    re = np.zeros(P.n // 2)
    im = np.zeros(P.n // 2)
    for i in range(cfg.C):
        f = rng.uniform(-1, 1, w * w)
        if i < x.shape[0]:
            img = f.reshape(w, w)
            img[:cfg.w0, :cfg.w0] = x[i]
            f = img.reshape(-1)
        re[i * ell:(i + 1) * ell] = f[rev] / val
        im[i * ell:(i + 1) * ell] = f[rev + ell] / val
    le = cfg.l_em
    return (o.encrypt(o.encode_pt(re, le, cfg.s_em), nonce),
            o.encrypt(o.encode_pt(im, le, cfg.s_em), nonce + 1))


def _cins_pixels(o, ct, w):
    z = o.decode_slots(o.decrypt(ct))
    ell = w * w // 2
    C = len(z) // ell
    return np.stack([E.encode(z[i * ell:(i + 1) * ell], w * w) for i in range(C)])


@pytest.fixture(scope="module")
def ds_setup():
    """N = 2^10 with the config-2 prime chain: w = 8 (C = 16 per ciphertext), two input
    ciphertexts (32 channels of 4 x 4) -> 64 channels of 2 x 2 at w = 4"""
    P = PP.Params(10, 24, 3, 60, 42, 60, h=192, n_p=7, boot_bits=48, n_boot=14)
    o = Oracle(P, 31)
    w0, w, f = 4, 8, 3
    C = P.n // (w * w)
    x = rng.random((2 * C, w0, w0))
    W = rng.normal(0, 0.1, (4 * C, 2 * C, f, f))
    cfg_in = BT.BootConfig(o, w, w0, C, stride=2)
    cfg_out = BT.BootConfig(o, w // 2, w0 // 2, 4 * C)
    rots = set(BT.block_rotations(o, None, cfg_in)) | set(BT.block_rotations(o, None, cfg_out))
    o.gen_conj_key()
    o.gen_relin_key()
    return dict(o=o, P=P, w0=w0, w=w, C=C, x=x, W=W, cfg_in=cfg_in, cfg_out=cfg_out, rots=rots)


def _conv_plans(o, d, scale_in):
    P, C, w = d["P"], d["C"], d["w"]
    plans = []
    for t in range(2):
        Wt = E.decompose_kernels(d["W"], C, t)
        plans.append(o.conv_plan(Wt, 4 * C, 4 * C, Wt.shape[2], w // 2, 1,
                                 (d["cfg_out"].delta0 * float(P.q[1])) / scale_in))
    return plans


def test_downsample_tail_and_decomposed_conv(ds_setup):
    """stride-2 tail (mask, Re + i Im, decomposition, S_{l/4<-1}) decodes to the real CinS of
    the polyphase images; the two decomposed BSGS convs + HAdd + rescale decode to the stride-2
    conv2d (Alg. 2 up to the sum of the decomposed convs)"""
    d = ds_setup
    o, P, w, w0, C, x = d["o"], d["P"], d["w"], d["w0"], d["C"], d["x"]
    cfg = d["cfg_in"]
    assert cfg.l_out == cfg.l_em - 2 - len(cfg.stoc)
    outs = []
    for t in range(2):
        re, im = _tail_inputs(o, cfg, x[t * C:(t + 1) * C], 10 + 2 * t)
        o.gen_rotation_keys(d["rots"])
        y = BT.stoc1(o, re, im, cfg)
        assert y.level == cfg.l_out
        pix = _cins_pixels(o, y, w // 2)
        want = np.stack([E.flatten_padded(v, w // 2) for v in E.decompose_images(x[t * C:(t + 1) * C])])
        assert np.abs(pix - want).max() < 1e-6
        outs.append(o.level_down(y, 1))
    plans = _conv_plans(o, d, outs[0].scale)
    o.gen_rotation_keys(sorted(set(plans[0].rotations(P.n // 2)) | set(plans[1].rotations(P.n // 2))))
    acc = o.add(o.bsgs(outs[0], plans[0]), o.bsgs(outs[1], plans[1]))
    acc = o.rescale(acc)
    assert acc.level == 0 and abs(acc.scale - d["cfg_out"].delta0) < 1e-6 * acc.scale
    C2, w2 = 4 * C, w // 2
    got = E.conv_output_from_coeffs(o.decode_coeffs(o.decrypt(acc)), C2, w2 * w2, C2, w2, w0 // 2)
    assert np.abs(got - E.conv2d_stride2(x, d["W"])).max() < 1e-6


def test_downsample_layer_one_bootstrap(ds_setup):
    """the whole Alg. 2 layer: the output (64 channels at w = 4) matches the FP64 stride-2 conv
    within 2^-12 after one bootstrap; a stride-1 conv followed by densify would bootstrap
    s^2 = 4 ciphertexts (4C channels of w^2 pixels)"""
    d = ds_setup
    o, P, w, w0, C, x = d["o"], d["P"], d["w"], d["w0"], d["C"], d["x"]
    cfg_in, cfg_out = d["cfg_in"], d["cfg_out"]
    ins = []
    for t in range(2):
        re, im = _tail_inputs(o, cfg_in, x[t * C:(t + 1) * C], 20 + 2 * t)
        o.gen_rotation_keys(d["rots"])
        ins.append(o.level_down(BT.stoc1(o, re, im, cfg_in), 1))
    plans = _conv_plans(o, d, ins[0].scale)
    o.gen_rotation_keys(sorted(set(plans[0].rotations(P.n // 2)) | set(plans[1].rotations(P.n // 2))))
    o.ops = {k: 0 for k in o.ops}
    out = BT.block_multi(o, ins, plans, cfg_out)
    assert o.ops["modraise"] == 1
    densify_boots = (4 * C * w * w) // P.n
    assert densify_boots == 4 * o.ops["modraise"]
    assert out.level == cfg_out.l_out
    pix = _cins_pixels(o, out, w // 2)
    ref = E.conv2d_stride2(x, d["W"])
    want = np.stack([E.flatten_padded(v, w // 2) for v in ref])
    assert np.abs(pix - want).max() < 2.0 ** -12
