"""Pins of the oracle's FP64 layer against the paper's identities.

Sec. 2.2 (slot / coefficient encodings), Sec. 2.3 (T = V P, Eq. 2, S-factorisation),
Sec. 3.1 (Theorem 1, partial DFT), Sec. 3.3.1 + Appendix A (real CinS, Eq. 5-6),
Sec. 3.2.2 (slice rotation), Sec. 4 (fusion with StoC2, Eq. 8), Fig. 1 (conv2d as a
1-D convolution of padded, flattened channels).
"""
import numpy as np
import pytest

from oracle import encoding as E

rng = np.random.default_rng(7)


def cvec(n):
    return rng.normal(size=n) + 1j * rng.normal(size=n)


@pytest.mark.parametrize("n", [8, 16, 64])
def test_fft_encoding_matches_paper_formula(n):
    z = cvec(n // 2)
    f = E.encode(z, n)
    assert np.allclose(f, E.encode_explicit(z, n), atol=1e-12)
    assert np.allclose(E.decode(f, n), E.decode_explicit(f, n), atol=1e-12)
    assert np.allclose(E.decode(f, n), z, atol=1e-12)


def test_slot_and_coefficient_products():
    """<m><m'> = <m (.) m'>_slot and <m><m'> = <m~ * m~'>_coeff (Sec. 2.2)"""
    n = 32
    z1, z2 = cvec(n // 2), cvec(n // 2)
    prod = E.negacyclic_conv(E.encode(z1, n), E.encode(z2, n))
    assert np.allclose(E.decode(prod, n), z1 * z2, atol=1e-11)
    m1, m2 = cvec(n // 2), cvec(n // 2)
    c = E.negacyclic_conv(E.coeff_encode(m1), E.coeff_encode(m2))
    # the product polynomial's coefficients are the negacyclic convolution; U = [V | iV]
    U, V = E.U_matrix(n), E.V_matrix(n)
    assert np.allclose(U, np.hstack([V, 1j * V]), atol=1e-12)
    assert np.allclose(E.decode(c, n), E.decode(E.coeff_encode(m1), n) * E.decode(E.coeff_encode(m2), n))


@pytest.mark.parametrize("n", [16, 64])
def test_special_dft_factorisation(n):
    m = n // 2
    T = E.T_matrix(m)
    assert np.allclose(T, E.V_matrix(n) @ E.P_matrix(m), atol=1e-12)          # T = V P
    half = E.T_matrix(m // 2)
    W = np.diag(E.W_diag(m // 2))
    I = np.eye(m // 2)
    Z = np.zeros_like(I)
    rec = np.block([[I, W], [I, -W]]) @ np.block([[half, Z], [Z, half]])
    assert np.allclose(T, rec, atol=1e-12)                                      # Eq. 2
    assert np.allclose(E.diag_to_dense(E.S_range(m, 1, m), m), T, atol=1e-12)   # S_{N/4}..S_1
    for levels in (1, 2, 3):
        acc = np.eye(m)
        for D, strides in E.ctos_groups(n, levels):
            acc = E.diag_to_dense(D, m) @ acc
            a0, step, count = E.ap_of_group(strides, m)
            assert set(D) <= {(a0 + step * i) % m for i in range(count)}
        assert np.allclose(acc, np.linalg.inv(T), atol=1e-12)                   # CtoS = T^-1


def test_theorem1_partial_dft():
    """S_{l<-1} m = (T_l m_0 | ... | T_l m_{C-1})"""
    n, ell = 64, 8
    m = n // 2
    x = cvec(m)
    lhs = E.diag_apply(E.S_range(ell, 1, m), x)
    rhs = np.concatenate([E.T_matrix(ell) @ x[i * ell:(i + 1) * ell] for i in range(m // ell)])
    assert np.allclose(lhs, rhs, atol=1e-12)
    # and S_{N/2<-l} S_{l<-1} = T_{N/2}
    both = E.diag_mul(E.S_range(m, ell, m), E.S_range(ell, 1, m), m)
    assert np.allclose(E.diag_to_dense(both, m), E.T_matrix(m), atol=1e-12)
    # StoC1 groups multiply back to S_{l<-1}
    acc = np.eye(m)
    for D, _ in E.stoc1_groups(n, ell, 2):
        acc = E.diag_to_dense(D, m) @ acc
    assert np.allclose(acc, E.diag_to_dense(E.S_range(ell, 1, m), m), atol=1e-12)


def test_real_cins_eq5_and_appendix_a():
    n, ell = 64, 4
    m = n // 2
    C = m // ell
    sl = rng.normal(size=(C, 2 * ell))
    folded = np.concatenate([E.fold(s) for s in sl])
    Pl = np.kron(np.eye(C), E.P_matrix(ell))
    lhs = E.diag_to_dense(E.S_range(ell, 1, m), m) @ Pl @ folded               # Eq. 5, first form
    assert np.allclose(lhs, E.real_cins_slots(sl), atol=1e-12)                  # second form
    for s in sl:
        assert np.allclose(E.dft_prime(s), E.dft_prime_explicit(s), atol=1e-12)
        y = rng.normal(size=2 * ell)
        # Appendix A: DFT'(x) (.) DFT'(y) = DFT'(x *_{2l} y)
        assert np.allclose(E.dft_prime(s) * E.dft_prime(y), E.dft_prime(E.negacyclic_conv(s, y)),
                           atol=1e-12)
    # Eq. 6: product of real-CinS plaintexts = slice-wise negacyclic convolution
    sl2 = rng.normal(size=(C, 2 * ell))
    prod = E.real_cins_slots(sl) * E.real_cins_slots(sl2)
    want = E.real_cins_slots(np.stack([E.negacyclic_conv(a, b) for a, b in zip(sl, sl2)]))
    assert np.allclose(prod, want, atol=1e-11)


def test_slice_rotation():
    """HRot by k*l rotates whole slices (Sec. 3.2.2)"""
    n, ell = 64, 4
    C = n // (2 * ell)
    sl = rng.normal(size=(C, 2 * ell))
    z = E.real_cins_slots(sl)
    for k in range(C):
        assert np.allclose(np.roll(z, -k * ell), E.real_cins_slots(np.roll(sl, -k, axis=0)))


def test_conv2d_as_negacyclic_convolution():
    """Fig. 1: zero-padded, flattened conv == 2-D cross-correlation at the real pixels"""
    for w0, f in ((4, 3), (5, 3), (8, 3), (6, 5)):
        w = E.pad_width(w0, f)
        x = rng.normal(size=(w0, w0))
        K = rng.normal(size=(f, f))
        out = E.negacyclic_conv(E.kernel_vector(K, w), E.flatten_padded(x, w)).reshape(w, w)
        ref = E.conv2d_same(x[None], K[None, None])[0]
        assert np.allclose(out[:w0, :w0], ref, atol=1e-12)


def test_fused_conv_layout():
    """S'K^ applied to a real-CinS input, read as coefficients, holds o_i at k*C + rev_C(i)
    (Sec. 4: conv fused with StoC2 ends coefficient-encoded; Thm. 2 with Y = X^C)"""
    n, w0, f = 256, 4, 3
    w = E.pad_width(w0, f)
    C = n // (w * w)
    cin, cout = 3, 4
    x = rng.normal(size=(cin, w0, w0))
    W = rng.normal(size=(cout, cin, f, f))
    z = E.cins_input_slots(x, w, n)
    diags = E.fused_conv_diagonals(W, cin, cout, f, w, n)
    ell = w * w // 2
    y = sum(d * np.roll(z, -k * ell) for k, d in enumerate(diags))            # Eq. 7 in slot view
    coeffs = E.encode(y, n)                                                     # slots -> polynomial
    got = E.conv_output_from_coeffs(coeffs, C, w * w, cout, w, w0)
    assert np.allclose(got, E.conv2d_same(x, W), atol=1e-10)
