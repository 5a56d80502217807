/*
 * oracle/ckks_ref.c -- integer primitives of the CPU oracle for RNS-CKKS.
 *
 * TEST INFRASTRUCTURE ONLY.  This file, like everything under oracle/, exists to
 * check the CUDA library; only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load it.  It shares no code,
 * header, table or constant generator with paper_2312_04356_gb300/.
 *
 * Everything here is written for obviousness, not speed: modular products use a
 * 128-bit product and the C '%' operator, NTTs are the textbook iterative
 * Cooley-Tukey / Gentleman-Sande loops, base conversion is the plain sum.  The
 * only concession to speed is an OpenMP loop over independent limbs.
 *
 * Ring and scheme: R_q = Z_q[X]/(X^N+1) (Sec. 2, "Preliminaries"); RNS-CKKS
 * (Sec. 2.1, which defers the formal scheme to the RNS-CKKS paper it cites).
 * Polynomials are stored limb-major: a[limb][coefficient], uint64 residues.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

/* threads of the OpenMP loops from now on (n >= 1) */
void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* threads the OpenMP loops over limbs use (1 without OpenMP) */
int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* scalar modular arithmetic (q < 2^62)                                */
/* ------------------------------------------------------------------ */
static inline u64 mul_mod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static inline u64 add_mod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static inline u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + (q - b); }

static u64 pow_mod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mul_mod(r, a, q);
        a = mul_mod(a, a, q);
        e >>= 1;
    }
    return r;
}
/* q prime: Fermat inverse */
static u64 inv_mod(u64 a, u64 q) { return pow_mod(a, q - 2, q); }

/* signed integer -> residue mod q */
static inline u64 from_signed(i64 v, u64 q) {
    if (v >= 0) return (u64)v % q;
    u64 m = (u64)(-(v + 1)) + 1; /* |v| without overflow */
    m %= q;
    return m == 0 ? 0 : q - m;
}

static unsigned bit_reverse(unsigned x, int bits) {
    unsigned r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

u64 orc_pow_mod(u64 a, u64 e, u64 q) { return pow_mod(a, e, q); }
u64 orc_mul_mod(u64 a, u64 b, u64 q) { return mul_mod(a, b, q); }

/* ------------------------------------------------------------------ */
/* negacyclic NTT                                                      */
/* ------------------------------------------------------------------ */
/*
 * Definition (the one every other routine here is pinned to):
 *   forward:  A[i] = sum_j a[j] * psi^((2*rev(i)+1)*j)   (mod q)
 * i.e. evaluation of a(X) at the odd powers of a primitive 2N-th root psi,
 * stored in bit-reversed order.  orc_ntt_naive computes exactly this sum.
 */
void orc_ntt_naive(const u64 *a, u64 *out, int logn, u64 q, u64 psi) {
    int n = 1 << logn;
    for (int i = 0; i < n; i++) {
        u64 root = pow_mod(psi, 2 * (u64)bit_reverse(i, logn) + 1, q);
        u64 acc = 0, pw = 1;
        for (int j = 0; j < n; j++) {
            acc = add_mod(acc, mul_mod(a[j], pw, q), q);
            pw = mul_mod(pw, root, q);
        }
        out[i] = acc;
    }
}

/* Cooley-Tukey, natural order in, bit-reversed order out. */
static void ntt_forward_one(u64 *a, int logn, u64 q, u64 psi) {
    int n = 1 << logn;
    u64 *tw = (u64 *)malloc(sizeof(u64) * n);
    for (int k = 0; k < n; k++) tw[k] = pow_mod(psi, bit_reverse(k, logn), q);
    for (int m = 1, t = n / 2; m < n; m *= 2, t /= 2) {
        for (int i = 0; i < m; i++) {
            u64 w = tw[m + i];
            int j1 = 2 * i * t;
            for (int j = j1; j < j1 + t; j++) {
                u64 u = a[j], v = mul_mod(a[j + t], w, q);
                a[j] = add_mod(u, v, q);
                a[j + t] = sub_mod(u, v, q);
            }
        }
    }
    free(tw);
}

/* Gentleman-Sande, bit-reversed order in, natural order out, times N^-1. */
static void ntt_inverse_one(u64 *a, int logn, u64 q, u64 psi) {
    int n = 1 << logn;
    u64 psi_inv = inv_mod(psi, q);
    u64 *tw = (u64 *)malloc(sizeof(u64) * n);
    for (int k = 0; k < n; k++) tw[k] = pow_mod(psi_inv, bit_reverse(k, logn), q);
    for (int m = n / 2, t = 1; m >= 1; m /= 2, t *= 2) {
        for (int i = 0; i < m; i++) {
            u64 w = tw[m + i];
            int j1 = 2 * i * t;
            for (int j = j1; j < j1 + t; j++) {
                u64 u = a[j], v = a[j + t];
                a[j] = add_mod(u, v, q);
                a[j + t] = mul_mod(sub_mod(u, v, q), w, q);
            }
        }
    }
    u64 n_inv = inv_mod((u64)n % q, q);
    for (int j = 0; j < n; j++) a[j] = mul_mod(a[j], n_inv, q);
    free(tw);
}

void orc_ntt_forward(u64 *a, int nlimbs, int logn, const u64 *q, const u64 *psi) {
    int n = 1 << logn;
#pragma omp parallel for schedule(dynamic)
    for (int l = 0; l < nlimbs; l++) ntt_forward_one(a + (size_t)l * n, logn, q[l], psi[l]);
}

void orc_ntt_inverse(u64 *a, int nlimbs, int logn, const u64 *q, const u64 *psi) {
    int n = 1 << logn;
#pragma omp parallel for schedule(dynamic)
    for (int l = 0; l < nlimbs; l++) ntt_inverse_one(a + (size_t)l * n, logn, q[l], psi[l]);
}

/* schoolbook product in Z_q[X]/(X^N+1): the definition NTT products are pinned to */
void orc_negacyclic_naive(const u64 *a, const u64 *b, u64 *out, int n, u64 q) {
    for (int k = 0; k < n; k++) out[k] = 0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            u64 p = mul_mod(a[i], b[j], q);
            int k = i + j;
            if (k < n) out[k] = add_mod(out[k], p, q);
            else out[k - n] = sub_mod(out[k - n], p, q);
        }
}

/* ------------------------------------------------------------------ */
/* limb-wise arithmetic on [nlimbs][n] arrays, modulus q[limb]          */
/* ------------------------------------------------------------------ */
void orc_add(const u64 *a, const u64 *b, u64 *o, int nl, int n, const u64 *q) {
#pragma omp parallel for
    for (int l = 0; l < nl; l++)
        for (int j = 0; j < n; j++) o[(size_t)l * n + j] = add_mod(a[(size_t)l * n + j], b[(size_t)l * n + j], q[l]);
}
void orc_sub(const u64 *a, const u64 *b, u64 *o, int nl, int n, const u64 *q) {
#pragma omp parallel for
    for (int l = 0; l < nl; l++)
        for (int j = 0; j < n; j++) o[(size_t)l * n + j] = sub_mod(a[(size_t)l * n + j], b[(size_t)l * n + j], q[l]);
}
void orc_neg(const u64 *a, u64 *o, int nl, int n, const u64 *q) {
#pragma omp parallel for
    for (int l = 0; l < nl; l++)
        for (int j = 0; j < n; j++) o[(size_t)l * n + j] = sub_mod(0, a[(size_t)l * n + j], q[l]);
}
/* pointwise product (used on NTT-domain data) */
void orc_mul(const u64 *a, const u64 *b, u64 *o, int nl, int n, const u64 *q) {
#pragma omp parallel for
    for (int l = 0; l < nl; l++)
        for (int j = 0; j < n; j++) o[(size_t)l * n + j] = mul_mod(a[(size_t)l * n + j], b[(size_t)l * n + j], q[l]);
}
/* o += a * b pointwise */
void orc_mul_acc(const u64 *a, const u64 *b, u64 *o, int nl, int n, const u64 *q) {
#pragma omp parallel for
    for (int l = 0; l < nl; l++)
        for (int j = 0; j < n; j++) {
            size_t k = (size_t)l * n + j;
            o[k] = add_mod(o[k], mul_mod(a[k], b[k], q[l]), q[l]);
        }
}
/* o = a * s[limb] (s already reduced mod q[limb]) */
void orc_mul_scalar(const u64 *a, const u64 *s, u64 *o, int nl, int n, const u64 *q) {
#pragma omp parallel for
    for (int l = 0; l < nl; l++)
        for (int j = 0; j < n; j++) o[(size_t)l * n + j] = mul_mod(a[(size_t)l * n + j], s[l] % q[l], q[l]);
}

/* reduce a vector of signed integers into every limb */
void orc_signed_to_rns(const i64 *v, u64 *o, int nl, int n, const u64 *q) {
#pragma omp parallel for
    for (int l = 0; l < nl; l++)
        for (int j = 0; j < n; j++) o[(size_t)l * n + j] = from_signed(v[j], q[l]);
}

/* ------------------------------------------------------------------ */
/* Galois automorphism X -> X^g in the coefficient domain               */
/* ------------------------------------------------------------------ */
/* a(X^g): coefficient i moves to i*g mod 2N, negated when that lands in [N,2N). */
void orc_automorphism(const u64 *a, u64 *o, int nl, int logn, const u64 *q, u64 g) {
    int n = 1 << logn;
    u64 two_n = 2 * (u64)n;
#pragma omp parallel for
    for (int l = 0; l < nl; l++) {
        const u64 *src = a + (size_t)l * n;
        u64 *dst = o + (size_t)l * n;
        for (int i = 0; i < n; i++) {
            u64 k = ((u64)i * g) % two_n;
            if (k < (u64)n) dst[k] = src[i];
            else dst[k - n] = sub_mod(0, src[i], q[l]);
        }
    }
}

/* ------------------------------------------------------------------ */
/* RNS base conversion (coefficient domain), no correction term         */
/* ------------------------------------------------------------------ */
/*
 * Input x given by residues x_i mod q_i (i < nin).  With Q = prod q_i and
 * Qhat_i = Q / q_i, output for each target modulus m:
 *     y_m = sum_i [ x_i * Qhat_i^{-1} ]_{q_i} * (Qhat_i mod m)   (mod m)
 * which equals x + u*Q (mod m) for some 0 <= u < nin.
 */
void orc_base_convert(const u64 *in, int nin, const u64 *qin, u64 *out, int nout, const u64 *qout, int n) {
    u64 *qhat_inv = (u64 *)malloc(sizeof(u64) * nin);
    u64 *qhat_mod = (u64 *)malloc(sizeof(u64) * (size_t)nin * nout);
    for (int i = 0; i < nin; i++) {
        u64 prod = 1;
        for (int k = 0; k < nin; k++)
            if (k != i) prod = mul_mod(prod, qin[k] % qin[i], qin[i]);
        qhat_inv[i] = inv_mod(prod, qin[i]);
        for (int m = 0; m < nout; m++) {
            u64 pm = 1;
            for (int k = 0; k < nin; k++)
                if (k != i) pm = mul_mod(pm, qin[k] % qout[m], qout[m]);
            qhat_mod[(size_t)i * nout + m] = pm;
        }
    }
#pragma omp parallel for
    for (int j = 0; j < n; j++) {
        for (int m = 0; m < nout; m++) {
            u64 acc = 0;
            for (int i = 0; i < nin; i++) {
                u64 xi = mul_mod(in[(size_t)i * n + j], qhat_inv[i], qin[i]);
                acc = add_mod(acc, mul_mod(xi % qout[m], qhat_mod[(size_t)i * nout + m], qout[m]), qout[m]);
            }
            out[(size_t)m * n + j] = acc;
        }
    }
    free(qhat_inv);
    free(qhat_mod);
}

/* ------------------------------------------------------------------ */
/* rescale, ModDown, ModRaise (coefficient domain)                      */
/* ------------------------------------------------------------------ */
/* centred representative of v mod qs, reduced into mod qt */
static inline u64 centred_to(u64 v, u64 qs, u64 qt) {
    if (v <= (qs >> 1)) return v % qt;
    u64 m = (qs - v) % qt; /* v - qs is negative, magnitude qs - v */
    return m == 0 ? 0 : qt - m;
}

/* Rescale (Sec. 2.4): c'_i = (c_i - [c_l]_{q_l, centred}) * q_l^{-1} mod q_i, i < l.
   in: [l+1][n], out: [l][n] */
void orc_rescale(const u64 *in, u64 *out, int l, int n, const u64 *q) {
    const u64 *last = in + (size_t)l * n;
    u64 ql = q[l];
#pragma omp parallel for
    for (int i = 0; i < l; i++) {
        u64 inv = inv_mod(ql % q[i], q[i]);
        for (int j = 0; j < n; j++) {
            u64 r = centred_to(last[j], ql, q[i]);
            out[(size_t)i * n + j] = mul_mod(sub_mod(in[(size_t)i * n + j], r, q[i]), inv, q[i]);
        }
    }
}

/* ModDown: in [nq+np][n] over Q u P (Q limbs first); out [nq][n]:
   out_i = (c_i - Conv_{P->q_i}([c]_P)) * P^{-1} mod q_i */
void orc_mod_down(const u64 *in, u64 *out, int nq, int np, int n, const u64 *q, const u64 *p) {
    u64 *conv = (u64 *)malloc(sizeof(u64) * (size_t)nq * n);
    orc_base_convert(in + (size_t)nq * n, np, p, conv, nq, q, n);
#pragma omp parallel for
    for (int i = 0; i < nq; i++) {
        u64 pinv = 1;
        for (int k = 0; k < np; k++) pinv = mul_mod(pinv, p[k] % q[i], q[i]);
        pinv = inv_mod(pinv, q[i]);
        for (int j = 0; j < n; j++)
            out[(size_t)i * n + j] = mul_mod(sub_mod(in[(size_t)i * n + j], conv[(size_t)i * n + j], q[i]), pinv, q[i]);
    }
    free(conv);
}

/* Exact rounded division by M = prod S_k (a ModDown by P fused with the rescale by q_l,
   Sec. 2.4): in rows 0..l-1 hold x mod q_i, rows l..l+nS-1 hold x mod S_k; out_i =
   round(x / M) mod q_i = (x_i - r) M^{-1} mod q_i with r the centred remainder of x mod M.
   r comes from the CRT written out in multi-precision integers: X = sum_k xhat_k (M / S_k),
   xhat_k = x_k (M / S_k)^{-1} mod S_k, is x mod M plus a multiple of M below nS M; subtract
   M until X < M, then r = X or X - M (whichever lies in (-M/2, M/2]). */
#define BIG_WORDS 10                      /* 640 bits: M up to 8 primes of 61 bits, X < 9 M */
typedef struct { u64 w[BIG_WORDS]; } big_t;

static void big_set(big_t *a, u64 v) { memset(a, 0, sizeof(*a)); a->w[0] = v; }
static void big_mul_word(big_t *a, u64 m) {          /* a *= m */
    u128 carry = 0;
    for (int i = 0; i < BIG_WORDS; i++) {
        u128 t = (u128)a->w[i] * m + carry;
        a->w[i] = (u64)t;
        carry = t >> 64;
    }
}
static void big_add_mul_word(big_t *a, const big_t *b, u64 m) {   /* a += b * m */
    u128 carry = 0;
    for (int i = 0; i < BIG_WORDS; i++) {
        u128 t = (u128)b->w[i] * m + a->w[i] + carry;
        a->w[i] = (u64)t;
        carry = t >> 64;
    }
}
static int big_cmp(const big_t *a, const big_t *b) {
    for (int i = BIG_WORDS - 1; i >= 0; i--)
        if (a->w[i] != b->w[i]) return a->w[i] > b->w[i] ? 1 : -1;
    return 0;
}
static void big_sub(big_t *a, const big_t *b) {      /* a -= b, a >= b */
    u64 borrow = 0;
    for (int i = 0; i < BIG_WORDS; i++) {
        u64 bi = b->w[i] + borrow;
        u64 nb = (bi < borrow) || (a->w[i] < bi);
        a->w[i] -= bi;
        borrow = nb;
    }
}
static u64 big_mod_word(const big_t *a, u64 q) {      /* a mod q, Horner over the words */
    u64 r = 0;
    for (int i = BIG_WORDS - 1; i >= 0; i--) r = (u64)((((u128)r << 64) | a->w[i]) % q);
    return r;
}

void orc_div_round(const u64 *in, u64 *out, int l, int nS, int n, const u64 *q, const u64 *S) {
    big_t M, Mk[16], Mhalf;
    u64 Mk_inv[16];
    big_set(&M, 1);
    for (int k = 0; k < nS; k++) big_mul_word(&M, S[k]);
    for (int k = 0; k < nS; k++) {
        u64 prod = 1;
        big_set(&Mk[k], 1);
        for (int t = 0; t < nS; t++)
            if (t != k) {
                big_mul_word(&Mk[k], S[t]);
                prod = mul_mod(prod, S[t] % S[k], S[k]);
            }
        Mk_inv[k] = inv_mod(prod, S[k]);
    }
    Mhalf = M;                                           /* floor(M / 2) */
    for (int i = 0; i < BIG_WORDS; i++)
        Mhalf.w[i] = (M.w[i] >> 1) | (i + 1 < BIG_WORDS ? M.w[i + 1] << 63 : 0);
    u64 *Mmod = (u64 *)malloc(sizeof(u64) * (size_t)(l + 1));
    u64 *Minv = (u64 *)malloc(sizeof(u64) * (size_t)(l + 1));
    for (int i = 0; i < l; i++) {
        Mmod[i] = big_mod_word(&M, q[i]);
        Minv[i] = inv_mod(Mmod[i], q[i]);
    }
#pragma omp parallel for
    for (int j = 0; j < n; j++) {
        big_t X;
        big_set(&X, 0);
        for (int k = 0; k < nS; k++) {
            u64 xk = in[(size_t)(l + k) * n + j];
            big_add_mul_word(&X, &Mk[k], mul_mod(xk, Mk_inv[k], S[k]));
        }
        while (big_cmp(&X, &M) >= 0) big_sub(&X, &M);
        int neg = big_cmp(&X, &Mhalf) > 0;               /* r = X - M */
        for (int i = 0; i < l; i++) {
            u64 rm = big_mod_word(&X, q[i]);
            if (neg) rm = sub_mod(rm, Mmod[i], q[i]);
            out[(size_t)i * n + j] = mul_mod(sub_mod(in[(size_t)i * n + j], rm, q[i]), Minv[i], q[i]);
        }
    }
    free(Mmod);
    free(Minv);
}

/* ModRaise (Sec. 2.4): the centred residue mod q0 lifted to every limb */
void orc_mod_raise(const u64 *in, u64 *out, int nq, int n, const u64 *q) {
#pragma omp parallel for
    for (int i = 0; i < nq; i++)
        for (int j = 0; j < n; j++) out[(size_t)i * n + j] = centred_to(in[j], q[0], q[i]);
}

/* ------------------------------------------------------------------ */
/* seeded randomness: SplitMix64 (Steele, Lea, Flood 2014) as a counter */
/* ------------------------------------------------------------------ */
#define SM_GAMMA 0x9E3779B97F4A7C15ULL
u64 orc_splitmix_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* key of one stream; the i-th word of the stream is the i-th SplitMix64 output from state `key` */
u64 orc_stream_key(u64 seed, u64 tag) { return orc_splitmix_mix(seed ^ orc_splitmix_mix(tag + SM_GAMMA)); }
static inline u64 stream_word(u64 key, u64 i) { return orc_splitmix_mix(key + (i + 1) * SM_GAMMA); }
u64 orc_stream_word(u64 key, u64 i) { return stream_word(key, i); }

/* uniform residues, drawn directly as NTT-domain values: limb with global prime id
   pid, slot j takes the 128-bit word (w[2k] << 64 | w[2k+1]) mod q, k = pid*n + j */
void orc_sample_uniform(u64 *out, int nl, int n, const u64 *q, const int *prime_id, u64 seed, u64 tag) {
    u64 key = orc_stream_key(seed, tag);
#pragma omp parallel for
    for (int l = 0; l < nl; l++)
        for (int j = 0; j < n; j++) {
            u64 k = (u64)prime_id[l] * (u64)n + (u64)j;
            u128 w = ((u128)stream_word(key, 2 * k) << 64) | stream_word(key, 2 * k + 1);
            out[(size_t)l * n + j] = (u64)(w % q[l]);
        }
}

/* uniform ternary {-1,0,1}: word mod 3, minus 1 */
void orc_sample_ternary(i64 *out, int n, u64 seed, u64 tag) {
    u64 key = orc_stream_key(seed, tag);
    for (int j = 0; j < n; j++) out[j] = (i64)(stream_word(key, j) % 3) - 1;
}

/* ternary with exactly h non-zeros: partial Fisher-Yates over positions, sign from a second stream */
void orc_sample_hw(i64 *out, int n, int h, u64 seed, u64 tag_pos, u64 tag_sign) {
    u64 kp = orc_stream_key(seed, tag_pos), ks = orc_stream_key(seed, tag_sign);
    int *perm = (int *)malloc(sizeof(int) * n);
    for (int j = 0; j < n; j++) { perm[j] = j; out[j] = 0; }
    for (int i = 0; i < h; i++) {
        int r = (int)(stream_word(kp, i) % (u64)(n - i));
        int t = perm[i]; perm[i] = perm[i + r]; perm[i + r] = t;
        out[perm[i]] = (stream_word(ks, i) & 1) ? -1 : 1;
    }
    free(perm);
}

/* discrete Gaussian, truncated to |e| <= 19 (6 sigma at sigma = 3.2), by cumulative table:
   weight(v) = exp(-(v*v) / (2 sigma^2)), v = -19..19; T[k] = floor(2^63 * cum_k / Z), T[38] = 2^63;
   sample = (smallest k with (word >> 1) < T[k]) - 19 */
#define GAUSS_BOUND 19
void orc_gauss_table(double sigma, u64 *table) {
    double w[2 * GAUSS_BOUND + 1], z = 0.0, cum = 0.0;
    for (int k = 0; k <= 2 * GAUSS_BOUND; k++) {
        int v = k - GAUSS_BOUND;
        w[k] = exp(-(double)(v * v) / (2.0 * sigma * sigma));
        z += w[k];
    }
    for (int k = 0; k <= 2 * GAUSS_BOUND; k++) {
        cum += w[k];
        table[k] = (u64)(cum / z * 9223372036854775808.0);
    }
    table[2 * GAUSS_BOUND] = 9223372036854775808ULL;
}
void orc_sample_gauss(i64 *out, int n, double sigma, u64 seed, u64 tag) {
    u64 table[2 * GAUSS_BOUND + 1];
    orc_gauss_table(sigma, table);
    u64 key = orc_stream_key(seed, tag);
    for (int j = 0; j < n; j++) {
        u64 u = stream_word(key, j) >> 1;
        int k = 0;
        while (u >= table[k]) k++;
        out[j] = (i64)k - GAUSS_BOUND;
    }
}
