"""FP64 encodings and linear maps of the oracle (plain numpy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Notation follows the paper:
  zeta = exp(pi i / N), zeta_j = zeta^(5^j), 0 <= j < N/2            (Sec. 2.2)
  U[j][k] = zeta_j^k ; slot encoding f = (1/N)(conj(U)^T m + U^T conj(m))  (Sec. 2.2)
  V[j][k] = zeta_j^k, k < N/2 ;  U = [V | i V]                           (Sec. 2.3)
  T_n[i][j] = omega_{4n}^(5^i * rev_n(j)) ; T_{N/2} = V P               (Sec. 2.3)
  T_n = [[I, W_{n/2}],[I, -W_{n/2}]] diag(T_{n/2}, T_{n/2}),  W_{n/2} = diag(omega_{4n}^(5^i))  (Eq. 2)
  S_k = blockdiag(B_k), B_k = [[I_k, W_k],[I_k, -W_k]], W_k = diag(omega_{8k}^(5^i)) ; T_{N/2} = S_{N/4}...S_1
  S_{j<-i} = S_{j/2} S_{j/4} ... S_i                                    (Sec. 3.1)
  real CinS: <m>_CinS = <S_{l<-1} P_l (check m_1 | ...)>_slot = <(DFT'_{2l}(m_i))_i>_slot  (Eq. 5)
  DFT'_{2l}(x)_j = sum_{k<2l} x_k omega_{4l}^(5^j k)                   (Appendix A)

Linear maps on the N/2 slots are kept as "diagonal dicts": {offset: vector} with
  (W m)_i = sum_offset d_offset[i] * m[(i + offset) mod M]               (Eq. 3)
"""
import numpy as np


# ---------------------------------------------------------------- basics ----
def bitrev_indices(n):
    bits = n.bit_length() - 1
    return np.array([int(format(i, "0%db" % bits)[::-1], 2) if bits else 0 for i in range(n)],
                    dtype=np.int64)


def rot_group(n_ring):
    """5^j mod 2N for j < N/2."""
    m = n_ring // 2
    out = np.empty(m, dtype=np.int64)
    g = 1
    for j in range(m):
        out[j] = g
        g = g * 5 % (2 * n_ring)
    return out


def omega(m, e):
    """omega_m^e = exp(2 pi i e / m) with e reduced mod m first (exact phase)."""
    e = np.asarray(e) % m
    return np.exp(2j * np.pi * e / m)


# ------------------------------------------------------- slot encoding -------
def U_matrix(n_ring):
    g = rot_group(n_ring)
    k = np.arange(n_ring)
    return omega(2 * n_ring, np.outer(g, k))


def encode_explicit(z, n_ring):
    """Sec. 2.2 formula, dense (small N only): f = (1/N)(conj(U)^T z + U^T conj(z))."""
    U = U_matrix(n_ring)
    f = (np.conj(U).T @ z + U.T @ np.conj(z)) / n_ring
    return f.real


def decode_explicit(f, n_ring):
    return U_matrix(n_ring) @ np.asarray(f, dtype=np.complex128)


def _odd_index(n_ring, e):
    """index m with 2m+1 = e (mod 2N), e odd."""
    return ((np.asarray(e) % (2 * n_ring)) - 1) // 2


def decode(f, n_ring):
    """z_j = sum_k f_k zeta^(5^j k): all odd-power evaluations by one FFT, then the 5^j ones."""
    k = np.arange(n_ring)
    tw = np.asarray(f, dtype=np.complex128) * omega(2 * n_ring, k)
    y = np.fft.ifft(tw) * n_ring           # y_m = f(zeta^(2m+1))
    return y[_odd_index(n_ring, rot_group(n_ring))]


def encode(z, n_ring):
    """Inverse of decode on real-coefficient polynomials (same result as encode_explicit)."""
    z = np.asarray(z, dtype=np.complex128)
    g = rot_group(n_ring)
    y = np.zeros(n_ring, dtype=np.complex128)
    y[_odd_index(n_ring, g)] = z
    y[_odd_index(n_ring, -g)] = np.conj(z)
    tw = np.fft.fft(y) / n_ring            # = f_k zeta^k
    k = np.arange(n_ring)
    return (tw * omega(2 * n_ring, -k)).real


def coeff_encode(m):
    """Coefficient encoding (Sec. 2.2): m in C^{N/2} -> (Re m | Im m)."""
    m = np.asarray(m, dtype=np.complex128)
    return np.concatenate([m.real, m.imag])


# ------------------------------------------------------ special DFT ---------
def V_matrix(n_ring):
    g = rot_group(n_ring)
    return omega(2 * n_ring, np.outer(g, np.arange(n_ring // 2)))


def T_matrix(n):
    """T_n[i][j] = omega_{4n}^(5^i rev_n(j))."""
    five = np.array([pow(5, i, 4 * n) for i in range(n)], dtype=np.int64)
    return omega(4 * n, np.outer(five, bitrev_indices(n)))


def P_matrix(n):
    P = np.zeros((n, n))
    P[np.arange(n), bitrev_indices(n)] = 1.0
    return P


def W_diag(k):
    """diagonal of W_k in B_k (the block of T_{2k} in Eq. 2, where W_{n/2} uses omega_{4n}):
    omega_{8k}^(5^i), i < k."""
    return np.array([omega(8 * k, pow(5, i, 8 * k)) for i in range(k)])


def S_factor(k, m, inverse=False):
    """S_k (or S_k^{-1}) on C^m as a diagonal dict.  B_k = [[I, W],[I, -W]],
    B_k^{-1} = (1/2)[[I, I],[W^{-1}, -W^{-1}]]."""
    w = W_diag(k)
    u = np.arange(m) % (2 * k)
    top = u < k
    wu = w[np.where(top, u, u - k)]
    d0 = np.zeros(m, dtype=np.complex128)
    dp = np.zeros(m, dtype=np.complex128)    # offset +k
    dm = np.zeros(m, dtype=np.complex128)    # offset -k
    if not inverse:
        d0[top] = 1.0
        dp[top] = wu[top]
        dm[~top] = 1.0
        d0[~top] = -wu[~top]
    else:
        d0[top] = 0.5
        dp[top] = 0.5
        dm[~top] = 0.5 / wu[~top]
        d0[~top] = -0.5 / wu[~top]
    out = {0: d0}
    if k % m:
        out[k % m] = out.get(k % m, 0) + dp
        out[(-k) % m] = out.get((-k) % m, 0) + dm
    else:
        out[0] = out[0] + dp + dm
    return out


def diag_mul(A, B, m):
    """(A B) as a diagonal dict: C_{a+b}[i] += A_a[i] * B_b[(i + a) mod m]."""
    C = {}
    for a, va in A.items():
        for b, vb in B.items():
            key = (a + b) % m
            term = va * np.roll(vb, -a)
            C[key] = C[key] + term if key in C else term
    return C


def diag_apply(D, x):
    """(D x)_i = sum_o d_o[i] x[(i + o) mod m]  (Eq. 3)."""
    out = np.zeros_like(np.asarray(x, dtype=np.complex128))
    for o, v in D.items():
        out += v * np.roll(x, -o)
    return out


def diag_to_dense(D, m):
    M = np.zeros((m, m), dtype=np.complex128)
    i = np.arange(m)
    for o, v in D.items():
        M[i, (i + o) % m] += v
    return M


def S_product(strides, m, inverse=False):
    """Product S_{strides[0]} S_{strides[1]} ... (left to right), as a diagonal dict."""
    out = {0: np.ones(m, dtype=np.complex128)}
    for k in strides:
        out = diag_mul(out, S_factor(k, m, inverse), m)
    return out


def S_range(j, i, m):
    """S_{j<-i} = S_{j/2} S_{j/4} ... S_i on C^m."""
    strides = []
    k = j // 2
    while k >= i:
        strides.append(k)
        k //= 2
    return S_product(strides, m)


def split_groups(stages, levels):
    """Split a list of stages into `levels` consecutive groups; the first groups take
    the extra stage when the count does not divide."""
    s = len(stages)
    base, extra = divmod(s, levels)
    out, pos = [], 0
    for g in range(levels):
        size = base + (1 if g < extra else 0)
        out.append(stages[pos: pos + size])
        pos += size
    return [grp for grp in out if grp]


def ctos_groups(n_ring, levels):
    """T_{N/2}^{-1} = S_1^{-1} ... S_{N/4}^{-1}: applied largest stride first, in `levels`
    groups.  Returns [(matrix diag dict, strides)] in application order."""
    m = n_ring // 2
    stages = [m >> (i + 1) for i in range(m.bit_length() - 1)]   # N/4, N/8, ..., 1
    groups = []
    for grp in split_groups(stages, levels):
        # group applies grp[0]^{-1} first: matrix = S_{grp[-1]}^{-1} ... S_{grp[0]}^{-1}
        groups.append((S_product(list(reversed(grp)), m, inverse=True), grp))
    return groups


def stoc1_groups(n_ring, ell, levels):
    """S_{ell<-1} = S_{ell/2} ... S_1 on C^{N/2}: applied S_1 first, in `levels` groups."""
    m = n_ring // 2
    stages = []
    k = 1
    while k < ell:
        stages.append(k)
        k *= 2
    groups = []
    for grp in split_groups(stages, levels):
        groups.append((S_product(list(reversed(grp)), m), grp))
    return groups


def ap_of_group(strides, m):
    """Diagonal offsets of a product of butterfly stages with strides k, 2k, ..., 2^(s-1)k
    form an arithmetic progression a0 + step*i, i < count (mod m)."""
    k = min(strides)
    s = len(strides)
    if (k << s) >= m:          # the offsets span every multiple of k
        return 0, k, m // k
    return (-((1 << s) - 1) * k) % m, k, (1 << (s + 1)) - 1


# ---------------------------------------------------------- real CinS -------
def dft_prime(x):
    """DFT'_{2l}(x)_j = sum_{k<2l} x_k omega_{4l}^(5^j k), j < l  (Appendix A)."""
    x = np.asarray(x, dtype=np.float64)
    two_l = x.shape[-1]
    return decode(x, two_l) if x.ndim == 1 else np.stack([decode(r, two_l) for r in x])


def dft_prime_explicit(x):
    x = np.asarray(x, dtype=np.float64)
    two_l = len(x)
    l = two_l // 2
    five = np.array([pow(5, j, 4 * l) for j in range(l)], dtype=np.int64)
    return omega(4 * l, np.outer(five, np.arange(two_l))) @ x


def fold(x):
    """check x_i = x_i + i x_{i+l} (Sec. 3.3.1)."""
    x = np.asarray(x, dtype=np.float64)
    l = len(x) // 2
    return x[:l] + 1j * x[l:]


def real_cins_slots(slices):
    """Slot vector of a real-CinS message: slices (C, 2l) -> concat_i DFT'_{2l}(m_i)."""
    slices = np.asarray(slices, dtype=np.float64)
    return np.concatenate([dft_prime(s) for s in slices])


def negacyclic_conv(x, y):
    """x *_{n} y in R[Y]/(Y^n + 1), n = len(x)."""
    n = len(x)
    full = np.convolve(x, y)
    out = full[:n].copy()
    out[: len(full) - n] -= full[n:]
    return out


# ---------------------------------------------------------- conv2d ----------
def pad_width(w0, f):
    """Padded image width: smallest power of two >= w0 + f//2 (zero border for 'same')."""
    w = 1
    while w < w0 + f // 2:
        w *= 2
    return w


def flatten_padded(img, w):
    """Zero-pad a (w0, w0) channel to (w, w) (data top-left) and flatten row-major."""
    w0 = img.shape[0]
    out = np.zeros((w, w))
    out[:w0, :w0] = img
    return out.reshape(-1)


def kernel_vector(K, w):
    """Length-w^2 vector k with (k *_{w^2} i)[p] = sum_{a,b} K[a,b] i[p + (a-c)w + (b-c)],
    i.e. PyTorch-style cross-correlation with 'same' padding.  A tap at offset -o < 0 is
    stored at w^2 - o with its sign flipped (Y^{-o} = -Y^{w^2 - o} in Y^{w^2} + 1)."""
    f = K.shape[0]
    c = f // 2
    n = w * w
    v = np.zeros(n)
    for a in range(f):
        for b in range(f):
            q = -((a - c) * w + (b - c))
            if q >= 0:
                v[q] += K[a, b]
            else:
                v[n + q] -= K[a, b]
    return v


def conv2d_same(x, W):
    """Plain FP64 cross-correlation, stride 1, zero 'same' padding: x (Cin, h, h), W (Cout, Cin, f, f)."""
    cin, h, _ = x.shape
    cout, _, f, _ = W.shape
    c = f // 2
    xp = np.zeros((cin, h + 2 * c, h + 2 * c))
    xp[:, c: c + h, c: c + h] = x
    out = np.zeros((cout, h, h))
    for o in range(cout):
        for i in range(cin):
            for a in range(f):
                for b in range(f):
                    out[o] += W[o, i, a, b] * xp[i, a: a + h, b: b + h]
    return out


def slice_matrix_of(D, C, ell):
    """C x C slice matrix of an ell-granular diagonal dict on C^{C*ell}:
    S'[i][j] = the length-ell block at rows i*ell.., columns j*ell.. (Eq. 8)."""
    S = np.zeros((C, C, ell), dtype=np.complex128)
    for o, v in D.items():
        assert o % ell == 0, "not ell-granular"
        d = o // ell
        for i in range(C):
            S[i, (i + d) % C] += v[i * ell: (i + 1) * ell]
    return S


def fused_conv_diagonals(W, cin, cout, f, w, n_ring):
    """Diagonals of K' = S' K^ (Sec. 4.2): the conv kernel matrix in slot view fused with
    StoC2 = S_{N/2<-l}.  Slice i of the ciphertext holds channel i (C = N/w^2 slices of
    2l = w^2 reals).  Returns [d_0, ..., d_{C-1}], d_delta[i l + u] = K'[i][(i+delta) % C][u]."""
    two_l = w * w
    ell = two_l // 2
    C = n_ring // two_l
    assert cin <= C and cout <= C
    Khat = np.zeros((C, C, ell), dtype=np.complex128)
    for o in range(cout):
        for i in range(cin):
            Khat[o, i] = dft_prime(kernel_vector(W[o, i], w))
    S = slice_matrix_of(S_range(n_ring // 2, ell, n_ring // 2), C, ell)
    Kp = np.einsum("imu,mju->iju", S, Khat)
    diags = []
    for d in range(C):
        v = np.zeros(n_ring // 2, dtype=np.complex128)
        for i in range(C):
            v[i * ell: (i + 1) * ell] = Kp[i, (i + d) % C]
        diags.append(v)
    return diags


def cins_input_slots(x, w, n_ring):
    """Real-CinS slot vector of an input feature map x (Cin, w0, w0): channel i in slice i."""
    two_l = w * w
    C = n_ring // two_l
    slices = np.zeros((C, two_l))
    for i in range(x.shape[0]):
        slices[i] = flatten_padded(x[i], w)
    return real_cins_slots(slices)


def conv_output_from_coeffs(coeff, C, two_l, cout, w, w0):
    """Read the fused conv output: coefficient k*C + rev_C(i) holds (o_i)_k (Thm. 2 with
    Y = X^C); returns (cout, w0, w0)."""
    rev = bitrev_indices(C) if C > 1 else np.array([0])
    out = np.zeros((cout, w0, w0))
    for i in range(cout):
        v = coeff[np.arange(two_l) * C + rev[i]]
        out[i] = v.reshape(w, w)[:w0, :w0]
    return out


# ---------------------------------------------------- depthwise conv2d -----
def dwconv_same(x, K):
    """FP64 depthwise cross-correlation, stride 1, zero 'same' padding: x (C, h, h), K (C, f, f)"""
    C, h, _ = x.shape
    f = K.shape[1]
    c = f // 2
    xp = np.zeros((C, h + 2 * c, h + 2 * c))
    xp[:, c: c + h, c: c + h] = x
    out = np.zeros((C, h, h))
    for i in range(C):
        for a in range(f):
            for b in range(f):
                out[i] += K[i, a, b] * xp[i, a: a + h, b: b + h]
    return out


def dwconv_kernel_slots(K, w, n_ring):
    """Sec. 3.3.4: the C kernels packed in one real-CinS plaintext <k_1 | ... | k_C>_CinS, so that
    one PMult gives k_i * i_i in every slice (Eq. 6)"""
    two_l = w * w
    C = n_ring // two_l
    slices = np.zeros((C, two_l))
    for i in range(K.shape[0]):
        slices[i] = kernel_vector(K[i], w)
    return real_cins_slots(slices)


# ------------------------------------------- downsampling conv2d (Alg. 2) -----
def G_matrix(w):
    """G_l of Appendix B, l = w^2/2: a 2w x 2w grid of (w/4 x w/4) blocks whose block (i, 2i) is
    the identity for i < w/2 and zero elsewhere.  (The appendix bounds i by <= w/2; a block at
    i = w/2 would write the slots that the j = 1 term of Alg. 2 fills, so the bound is strict.)"""
    ell = w * w // 2
    b = w // 4
    G = np.zeros((ell, ell))
    for i in range(w // 2):
        G[i * b:(i + 1) * b, 2 * i * b:(2 * i + 1) * b] = np.eye(b)
    return G


def blockdiag_to_diag(Gb, m):
    """diag(Gb, Gb, ...) on C^m as a diagonal dict"""
    ell = Gb.shape[0]
    D = {}
    rows, cols = np.nonzero(Gb)
    for r, c in zip(rows, cols):
        o = int(c - r) % m
        if o not in D:
            D[o] = np.zeros(m, dtype=np.complex128)
        D[o][r::ell] += Gb[r, c]
    return D


def rotation_diag(r, m):
    """ct << r, i.e. rot(z, r)_j = z_{j+r}, as a diagonal dict (ct >> r is r -> -r)"""
    return {r % m: np.ones(m, dtype=np.complex128)}


def decompose_diag(w, n_ring):
    """Alg. 2's decomposition as one linear map on the slots:
    D = sum_{j<4} (>> j l/4) calG_l (<< r_j),  r = (0, l/2, w/4, l/2 + w/4)"""
    m = n_ring // 2
    ell = w * w // 2
    G = blockdiag_to_diag(G_matrix(w), m)
    r = [0, ell // 2, w // 4, ell // 2 + w // 4]
    D = {}
    for j in range(4):
        t = diag_mul(rotation_diag(-j * (ell // 4), m), diag_mul(G, rotation_diag(r[j], m), m), m)
        for o, v in t.items():
            D[o] = D[o] + v if o in D else v
    return D


def decompose_ap(w, n_ring):
    """the offsets of decompose_diag: b w/4 for 1 - w <= b <= w - 1 -> (a0, step, count)"""
    m = n_ring // 2
    return ((1 - w) * (w // 4)) % m, w // 4, 2 * w - 1


def decompose_source(w, n_ring):
    """The same permutation from the layouts alone.  Slot i l + rev_l(k) holds pixels k and
    k + l of channel i (k = r w + c, r < w/2).  The polyphase image (p, q) of channel i,
    x_pq[u][v] = x[2u + p][2v + q] (w/2 x w/2), becomes slice 4i + q + 2p of length l/4, whose
    slot rev_{l/4}(u w/2 + v) holds its pixels (u, v) and (u + w/4, v).
    Returns src with new[x] = old[src[x]]."""
    m = n_ring // 2
    ell = w * w // 2
    l4 = ell // 4
    rev_l = bitrev_indices(ell)
    rev_4 = bitrev_indices(l4)
    src = np.full(m, -1, dtype=np.int64)
    for i in range(m // ell):
        for p in range(2):
            for q in range(2):
                for u in range(w // 4):
                    for v in range(w // 2):
                        k = (2 * u + p) * w + 2 * v + q
                        src[(4 * i + q + 2 * p) * l4 + rev_4[u * (w // 2) + v]] = i * ell + rev_l[k]
    return src


def decompose_images(x):
    """the polyphase images of x (C, h, h), h even: (4C, h/2, h/2), image 4i + q + 2p = x_i[p::2, q::2]"""
    C, h, _ = x.shape
    out = np.zeros((4 * C, h // 2, h // 2))
    for i in range(C):
        for p in range(2):
            for q in range(2):
                out[4 * i + q + 2 * p] = x[i, p::2, q::2]
    return out


def conv2d_stride2(x, W):
    """FP64 cross-correlation, stride 2, zero padding f//2 (PyTorch semantics), h even:
    out[o][y][x] = sum W[o,i,a,b] x[i][2y + a - c][2x + b - c]"""
    return conv2d_same(x, W)[:, ::2, ::2]


def decompose_kernels(W, C, t):
    """Alg. 2's decomposed kernels for input ciphertext t (channels tC .. tC + C - 1): the stride-2
    conv as a unit-stride conv over the polyphase images.  Tap (a, b) of W[o][tC + i] goes to
    slice 4i + q + 2p at offset (dy, dx), a - c = 2 dy + p, b - c = 2 dx + q; the result is a
    centred kernel of size 2R + 1, R = (c + 1) // 2.  Returns (cout, 4C, 2R + 1, 2R + 1)."""
    cout, cin, f, _ = W.shape
    c = f // 2
    R = (c + 1) // 2
    out = np.zeros((cout, 4 * C, 2 * R + 1, 2 * R + 1))
    for i in range(C):
        ch = t * C + i
        if ch >= cin:
            break
        for a in range(f):
            for b in range(f):
                p, q = (a - c) % 2, (b - c) % 2
                dy, dx = (a - c - p) // 2, (b - c - q) // 2
                out[:, 4 * i + q + 2 * p, dy + R, dx + R] += W[:, ch, a, b]
    return out


# ------------------------------------------------- FC fused with StoC (Sec. 4.3) -----
def fc_stoc_matrix(M, n_ring):
    """F = V M: the FC weights M (n_out x n_in) followed by the whole StoC.  With slot encoding
    (CinS with l = 1) the StoC takes the slot vector V y to the coefficient encoding of y
    (coefficients y_k, k < N/2), so HMatmul(F) on slots holding x leaves M x in the
    coefficients.  Column j of F = slots of the real polynomial with coefficients M[:, j]."""
    n_out, n_in = M.shape
    F = np.zeros((n_ring // 2, n_in), dtype=np.complex128)
    for j in range(n_in):
        f = np.zeros(n_ring)
        f[:n_out] = M[:, j]
        F[:, j] = decode(f, n_ring)
    return F


def fc_stoc_diagonals(M, n_ring):
    """diagonals of F acting on x replicated with period n_in (x_rep[j] = x[j mod n_in]):
    d_o[i] = F[i][(i + o) mod n_in], o < n_in (a0 = 0, step 1, count n_in)"""
    F = fc_stoc_matrix(M, n_ring)
    m, n_in = F.shape
    i = np.arange(m)
    return {o: F[i, (i + o) % n_in] for o in range(n_in)}
