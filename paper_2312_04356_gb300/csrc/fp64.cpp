// FP64 side of the library: canonical embedding, the factors of the special DFT,
// real CinS, fused conv diagonals, Chebyshev interpolation.  Offline (plaintext
// preparation) and client-side (encode/decode) work only.
//
//   slots   z_j = f(zeta^(5^j)), zeta = exp(pi i / N), j < N/2                (Sec. 2.2)
//   T_n     T_n[i][j] = omega_{4n}^(5^i rev_n(j)), T_{N/2} = S_{N/4} ... S_1    (Sec. 2.3, Eq. 2)
//   S_k     blockdiag(B_k), B_k = [[I, W_k], [I, -W_k]], W_k = diag(omega_{8k}^(5^i))
//   DFT'    DFT'_{2l}(x)_j = sum_{k<2l} x_k omega_{4l}^(5^j k)                 (Appendix A)
// A linear map on the N/2 slots is a map offset -> vector with
//   (W m)_i = sum_o d_o[i] m[(i + o) mod M]                                      (Eq. 3)
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace fp64 {

static const double PI = 3.14159265358979323846;

static cplx root_of_unity(long long e, long long m) {
    // exp(2 pi i e / m) with e reduced into [0, m)
    e %= m;
    if (e < 0) e += m;
    double th = 2.0 * PI * (double)e / (double)m;
    return cplx(cos(th), sin(th));
}

// in-place iterative radix-2 FFT; sign -1: sum_k a_k e^{-2 pi i jk/n}, sign +1: e^{+...}
static void fft(std::vector<cplx>& a, int sign) {
    const int n = (int)a.size();
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (int len = 2; len <= n; len <<= 1) {
        std::vector<cplx> w(len / 2);
        for (int k = 0; k < len / 2; ++k) w[k] = root_of_unity(sign * (long long)k, len);
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < len / 2; ++k) {
                cplx u = a[i + k], v = a[i + k + len / 2] * w[k];
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

static std::vector<long long> rot_group(int n) {
    std::vector<long long> g(n / 2);
    long long x = 1;
    for (int j = 0; j < n / 2; ++j) {
        g[j] = x;
        x = x * 5 % (2LL * n);
    }
    return g;
}

// index m with 2m + 1 = e (mod 2N)
static inline int odd_index(long long e, int n) {
    e %= 2LL * n;
    if (e < 0) e += 2LL * n;
    return (int)((e - 1) / 2);
}

std::vector<cplx> decode_slots(const std::vector<double>& f, int n) {
    // y_m = f(zeta^(2m+1)) = sum_k (f_k zeta^k) e^{2 pi i m k / N}
    std::vector<cplx> g(n);
    for (int k = 0; k < n; ++k) g[k] = f[k] * root_of_unity(k, 2LL * n);
    fft(g, +1);
    std::vector<long long> rg = rot_group(n);
    std::vector<cplx> z(n / 2);
    for (int j = 0; j < n / 2; ++j) z[j] = g[odd_index(rg[j], n)];
    return z;
}

std::vector<double> encode_slots(const std::vector<cplx>& z, int n) {
    // values at zeta^(5^j) are z_j, at zeta^(-5^j) their conjugates; invert the evaluation
    std::vector<cplx> y(n, cplx(0, 0));
    std::vector<long long> rg = rot_group(n);
    for (int j = 0; j < n / 2; ++j) {
        y[odd_index(rg[j], n)] = z[j];
        y[odd_index(-rg[j], n)] = std::conj(z[j]);
    }
    fft(y, -1);
    std::vector<double> f(n);
    for (int k = 0; k < n; ++k) f[k] = (y[k] / (double)n * root_of_unity(-(long long)k, 2LL * n)).real();
    return f;
}

// ------------------------------------------------------------- S factors ----
static std::vector<cplx> w_diag(int k) {
    std::vector<cplx> w(k);
    long long e = 1;
    for (int i = 0; i < k; ++i) {
        w[i] = root_of_unity(e, 8LL * k);
        e = e * 5 % (8LL * k);
    }
    return w;
}

static void acc_into(Diag& D, int off, const std::vector<cplx>& v) {
    auto it = D.find(off);
    if (it == D.end())
        D[off] = v;
    else
        for (size_t i = 0; i < v.size(); ++i) it->second[i] += v[i];
}

static Diag s_factor(int k, int m, bool inverse) {
    std::vector<cplx> w = w_diag(k);
    std::vector<cplx> d0(m), dp(m), dm(m);
    for (int i = 0; i < m; ++i) {
        int u = i % (2 * k);
        bool top = u < k;
        cplx wu = w[top ? u : u - k];
        if (!inverse) {
            if (top) {
                d0[i] = 1.0;
                dp[i] = wu;
            } else {
                dm[i] = 1.0;
                d0[i] = -wu;
            }
        } else {
            if (top) {
                d0[i] = 0.5;
                dp[i] = 0.5;
            } else {
                dm[i] = 0.5 / wu;
                d0[i] = -0.5 / wu;
            }
        }
    }
    Diag D;
    D[0] = d0;
    acc_into(D, k % m, dp);
    acc_into(D, ((-k) % m + m) % m, dm);
    return D;
}

static Diag diag_mul(const Diag& A, const Diag& B, int m) {
    Diag C;
    for (const auto& a : A)
        for (const auto& b : B) {
            int key = (a.first + b.first) % m;
            std::vector<cplx> t(m);
            for (int i = 0; i < m; ++i) t[i] = a.second[i] * b.second[(i + a.first) % m];
            acc_into(C, key, t);
        }
    return C;
}

Diag s_product(const std::vector<int>& strides, int m, bool inverse) {
    Diag out;
    out[0] = std::vector<cplx>(m, cplx(1, 0));
    for (int k : strides) out = diag_mul(out, s_factor(k, m, inverse), m);
    return out;
}

std::vector<std::vector<int>> split_groups(const std::vector<int>& stages, int levels) {
    std::vector<std::vector<int>> out;
    int s = (int)stages.size();
    int base = s / levels, extra = s % levels, pos = 0;
    for (int g = 0; g < levels; ++g) {
        int size = base + (g < extra ? 1 : 0);
        if (size > 0) out.push_back(std::vector<int>(stages.begin() + pos, stages.begin() + pos + size));
        pos += size;
    }
    return out;
}

void ap_of_group(const std::vector<int>& strides, int m, int* a0, int* step, int* count) {
    int k = *std::min_element(strides.begin(), strides.end());
    int s = (int)strides.size();
    if (((long long)k << s) >= m) {
        *a0 = 0;
        *step = k;
        *count = m / k;
    } else {
        *a0 = (int)((((long long)-((1LL << s) - 1) * k) % m + m) % m);
        *step = k;
        *count = (1 << (s + 1)) - 1;
    }
}

int default_bsgs_B(int count) {
    // 2^e with e the least integer such that 4^e >= count, i.e. 2^ceil(log2(count)/2)
    if (count <= 1) return 1;
    int e = 0;
    while ((1LL << (2 * e)) < count) ++e;
    return 1 << e;
}

// Bootstrapping HMatmuls are double hoisted: a baby step costs one key-switch inner product,
// a giant step about five (ModDown of c1, ModUp, inner product).  B = the power of two that
// minimises (B - 1) + 5 (G - 1), G = ceil(count / B); the smaller one on ties.
int boot_bsgs_B(int count) {
    long long best = -1;
    int bestB = 1;
    for (int B = 1;; B *= 2) {
        const long long G = (count + B - 1) / B;
        const long long cost = (B - 1) + 5 * (G - 1);
        if (best < 0 || cost < best) {
            best = cost;
            bestB = B;
        }
        if (B >= count) return bestB;
    }
}

// --------------------------------------------------------------- CinS ------
std::vector<cplx> real_cins_slots(const double* m, int C, int two_l) {
    const int ell = two_l / 2;
    std::vector<cplx> z((size_t)C * ell);
    for (int i = 0; i < C; ++i) {
        std::vector<double> sl(m + (size_t)i * two_l, m + (size_t)(i + 1) * two_l);
        std::vector<cplx> d = decode_slots(sl, two_l);   // DFT'_{2l}: the subring's embedding
        std::copy(d.begin(), d.end(), z.begin() + (size_t)i * ell);
    }
    return z;
}

std::vector<double> cins_to_reals(const std::vector<cplx>& z, int C, int two_l) {
    const int ell = two_l / 2;
    std::vector<double> out((size_t)C * two_l);
    for (int i = 0; i < C; ++i) {
        std::vector<cplx> sl(z.begin() + (size_t)i * ell, z.begin() + (size_t)(i + 1) * ell);
        std::vector<double> f = encode_slots(sl, two_l);
        std::copy(f.begin(), f.end(), out.begin() + (size_t)i * two_l);
    }
    return out;
}

// Fig. 1 placement: (k *_{w^2} i)[p] = sum_{a,b} K[a][b] i[p + (a-c) w + (b-c)]; a tap at
// offset -o < 0 goes to w^2 - o with its sign flipped (Y^{-o} = -Y^{w^2-o})
static std::vector<double> kernel_vector(const double* K, int f, int w) {
    const int c = f / 2, n = w * w;
    std::vector<double> v(n, 0.0);
    for (int a = 0; a < f; ++a)
        for (int b = 0; b < f; ++b) {
            int qo = -((a - c) * w + (b - c));
            if (qo >= 0)
                v[qo] += K[a * f + b];
            else
                v[n + qo] -= K[a * f + b];
        }
    return v;
}

// Sec. 3.3.4: the C depthwise kernels packed as one real-CinS slot vector <k_1 | ... | k_C>
std::vector<cplx> dwconv_kernel_slots(const double* K, int c, int f, int w, int n) {
    const int two_l = w * w, C = n / two_l;
    CK_CHECK(c >= 1 && c <= C, CKKS_EINVAL, "channels do not fit in one ciphertext");
    std::vector<double> m((size_t)C * two_l, 0.0);
    for (int i = 0; i < c; ++i) {
        std::vector<double> v = kernel_vector(K + (size_t)i * f * f, f, w);
        std::copy(v.begin(), v.end(), m.begin() + (size_t)i * two_l);
    }
    return real_cins_slots(m.data(), C, two_l);
}

// ------------------------------------------- downsampling conv2d (Alg. 2) ---
static int bit_reverse(int x, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

// Alg. 2's decomposition is a permutation of the slots.  Before it, slot
// i l + rev_l(k) holds pixels k and k + l of channel i (k = r w + c with r < w/2).  The
// polyphase image (p, q) of channel i, x[2u + p][2v + q] of size (w/2)^2, goes to slice
// 4i + q + 2p of length l/4, whose slot rev_{l/4}(u w/2 + v) holds its pixels (u, v) and
// (u + w/4, v).  The nonzero diagonals (0/1 masks) sit at offsets b w/4, |b| < w.
Diag decompose_diag(int w, int m) {
    const int ell = w * w / 2, l4 = ell / 4;
    int lb = 0, l4b = 0;
    while ((1 << lb) < ell) ++lb;
    while ((1 << l4b) < l4) ++l4b;
    Diag D;
    for (int i = 0; i < m / ell; ++i)
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q)
                for (int u = 0; u < w / 4; ++u)
                    for (int v = 0; v < w / 2; ++v) {
                        const int k = (2 * u + p) * w + 2 * v + q;
                        const long long dst = (long long)(4 * i + q + 2 * p) * l4 + bit_reverse(u * (w / 2) + v, l4b);
                        const long long src = (long long)i * ell + bit_reverse(k, lb);
                        const int off = (int)(((src - dst) % m + m) % m);
                        std::vector<cplx>& d = D[off];
                        if (d.empty()) d.assign(m, cplx(0, 0));
                        d[dst] = cplx(1, 0);
                    }
    return D;
}

// The stride-2 conv W[cout][cin][f][f] over input ciphertext t (channels tC .. tC + C - 1) as
// a unit-stride conv over their polyphase images: tap (a, b) of W[o][tC + i] becomes tap
// (dy + R, dx + R) of the kernel on slice 4i + q + 2p, with a - f/2 = 2 dy + p and
// b - f/2 = 2 dx + q, R = (f/2 + 1) / 2.  Returns W'[cout][4C][2R + 1][2R + 1].
std::vector<double> decompose_kernels(const double* W, int cout, int cin, int f, int C, int t, int* f_out) {
    const int c = f / 2, R = (c + 1) / 2, fo = 2 * R + 1;
    std::vector<double> out((size_t)cout * 4 * C * fo * fo, 0.0);
    for (int i = 0; i < C && t * C + i < cin; ++i)
        for (int a = 0; a < f; ++a)
            for (int b = 0; b < f; ++b) {
                const int p = ((a - c) % 2 + 2) % 2, q = ((b - c) % 2 + 2) % 2;
                const int dy = (a - c - p) / 2, dx = (b - c - q) / 2;
                const int slice = 4 * i + q + 2 * p;
                for (int o = 0; o < cout; ++o)
                    out[(((size_t)o * 4 * C + slice) * fo + dy + R) * fo + dx + R] +=
                        W[(((size_t)o * cin + t * C + i) * f + a) * f + b];
            }
    *f_out = fo;
    return out;
}

// FC fused with the whole StoC (Sec. 4.3; slot encoding is CinS with l = 1): F = V M, whose
// column j holds the slots of the real polynomial with coefficients M[:, j] (the StoC takes
// slots V y to coefficients y).  On x replicated with period n_in the product needs only
// the n_in diagonals d_o[i] = F[i][(i + o) mod n_in].
Diag fc_stoc_diagonals(const double* M, int n_out, int n_in, int n) {
    const int m = n / 2;
    std::vector<std::vector<cplx>> F(n_in);
    for (int j = 0; j < n_in; ++j) {
        std::vector<double> f(n, 0.0);
        for (int k = 0; k < n_out; ++k) f[k] = M[(size_t)k * n_in + j];
        F[j] = decode_slots(f, n);
    }
    Diag D;
    for (int o = 0; o < n_in; ++o) {
        std::vector<cplx> d(m);
        for (int i = 0; i < m; ++i) d[i] = F[(i + o) % n_in][i];
        D[o] = std::move(d);
    }
    return D;
}

std::vector<std::vector<cplx>> fused_conv_diagonals(const double* W, int cin, int cout, int f, int w, int n) {
    const int two_l = w * w, ell = two_l / 2, C = n / two_l, m = n / 2;
    CK_CHECK(C >= 1 && cin <= C && cout <= C, CKKS_EINVAL, "channels do not fit in one ciphertext");
    // K^[o][i] = DFT'_{2l}(k_{o,i})
    std::vector<std::vector<cplx>> Kh((size_t)C * C);
    for (int o = 0; o < cout; ++o)
        for (int i = 0; i < cin; ++i)
            Kh[(size_t)o * C + i] = decode_slots(kernel_vector(W + ((size_t)o * cin + i) * f * f, f, w), two_l);
    // S' = slice matrix of StoC2 = S_{N/2 <- l} = S_{N/4} ... S_l
    std::vector<int> strides;
    for (int k = m / 2; k >= ell; k /= 2) strides.push_back(k);
    Diag S = s_product(strides, m, false);
    std::vector<std::vector<cplx>> Sp((size_t)C * C, std::vector<cplx>(ell, cplx(0, 0)));
    for (const auto& d : S) {
        CK_CHECK(d.first % ell == 0, CKKS_EINVAL, "StoC2 is not slice-granular");
        int dd = d.first / ell;
        for (int i = 0; i < C; ++i)
            for (int u = 0; u < ell; ++u) Sp[(size_t)i * C + (i + dd) % C][u] += d.second[(size_t)i * ell + u];
    }
    // K' = S' K^ (slice-wise products), diagonal delta: d[i l + u] = K'[i][(i + delta) % C][u]
    std::vector<std::vector<cplx>> diags(C, std::vector<cplx>(m, cplx(0, 0)));
    for (int i = 0; i < C; ++i)
        for (int j = 0; j < C; ++j) {
            std::vector<cplx> acc(ell, cplx(0, 0));
            for (int mm = 0; mm < C; ++mm) {
                const std::vector<cplx>& kk = Kh[(size_t)mm * C + j];
                if (kk.empty()) continue;
                const std::vector<cplx>& ss = Sp[(size_t)i * C + mm];
                for (int u = 0; u < ell; ++u) acc[u] += ss[u] * kk[u];
            }
            int delta = ((j - i) % C + C) % C;
            for (int u = 0; u < ell; ++u) diags[delta][(size_t)i * ell + u] = acc[u];
        }
    return diags;
}

// Chebyshev interpolant (first-kind nodes) of cos(2 pi (K y - 1/4) / 2^r) on [-1, 1]
std::vector<double> cheb_interp_cos(double K, int r, int deg) {
    const int n = deg + 1;
    std::vector<double> fx(n), c(n, 0.0);
    for (int j = 0; j < n; ++j) {
        double x = cos(PI * (j + 0.5) / n);
        fx[j] = cos(2.0 * PI * (K * x - 0.25) / ldexp(1.0, r));
    }
    for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += fx[j] * cos(PI * k * (j + 0.5) / n);
        c[k] = 2.0 * s / n;
    }
    c[0] *= 0.5;
    return c;
}

// Power coefficients of p(x), x = (y - beta) / alpha, re-expressed as a Chebyshev series in y:
// the binomial change of variable, then Horner's rule in the Chebyshev basis (y T_0 = T_1,
// y T_j = (T_(j+1) + T_(j-1)) / 2).
std::vector<double> power_to_cheb(const std::vector<double>& c, double alpha, double beta) {
    const int n = (int)c.size();
    std::vector<double> py(n, 0.0);
    for (int k = 0; k < n; ++k) {
        double binom = 1.0;                                  // C(k, j), j = 0 .. k
        for (int j = 0; j <= k; ++j) {
            py[j] += c[k] * binom * std::pow(-beta, k - j) / std::pow(alpha, k);
            binom = binom * (k - j) / (j + 1);
        }
    }
    std::vector<double> r(1, py[n - 1]);
    for (int k = n - 2; k >= 0; --k) {
        std::vector<double> t(r.size() + 1, 0.0);            // y * r
        for (size_t j = 0; j < r.size(); ++j) {
            if (j == 0) {
                t[1] += r[0];
            } else {
                t[j + 1] += 0.5 * r[j];
                t[j - 1] += 0.5 * r[j];
            }
        }
        t[0] += py[k];
        r.swap(t);
    }
    r.resize(n);
    return r;
}

}  // namespace fp64
