// Host arithmetic and the RNS prime chain.
//
// Chain rule (the paper fixes N, L, dnum, Delta, h in Table 3 and is silent on
// the primes): q_0 is the largest prime < 2^q0_bits with q = 1 mod 2N; the
// special primes are the next largest below 2^p_bits; scaling primes are chosen
// top-down inside each segment (bootstrapping levels first, then circuit levels)
// as the unused prime = 1 mod 2N nearest to Delta_l^2 / 2^b, with Delta_top = 2^b
// and Delta_{l-1} = Delta_l^2 / q_l, so that rescaling a product of two level-l
// ciphertexts lands on the canonical scale of level l-1 (Sec. 2.4).
#include <math.h>

#include <algorithm>
#include <set>

#include "internal.h"

typedef unsigned __int128 u128;

namespace hostmath {

u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

u64 powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }

u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

u64 from_signed(int64_t v, u64 q) {
    if (v >= 0) return (u64)v % q;
    u64 m = ((u64)(-(v + 1)) + 1) % q;
    return m ? q - m : 0;
}

DevMod make_mod(u64 q) {
    DevMod m;
    m.q = q;
    int s = 0;
    while ((q >> s) != 0) ++s;
    m.s = s;
    m.mu = (u64)(((u128)1 << (2 * s)) / q);
    return m;
}

bool is_prime(u64 n) {
    if (n < 2) return false;
    static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : small)
        if (n % p == 0) return n == p;
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++s;
    }
    for (u64 a : small) {
        u64 x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < s; ++i) {
            x = mulmod(x, x, n);
            if (x == n - 1) {
                comp = false;
                break;
            }
        }
        if (comp) return false;
    }
    return true;
}

u64 splitmix_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
u64 stream_key(u64 seed, u64 tag) { return splitmix_mix(seed ^ splitmix_mix(tag + 0x9E3779B97F4A7C15ULL)); }
u64 stream_word(u64 key, u64 i) { return splitmix_mix(key + (i + 1) * 0x9E3779B97F4A7C15ULL); }

long long llround_away(double x) { return llround(x); }

}  // namespace hostmath

using namespace hostmath;

static std::vector<u64> largest_primes(int bits, u64 two_n, int count, const std::set<u64>& exclude) {
    std::vector<u64> out;
    u64 top = (bits >= 64) ? ~0ULL : ((1ULL << bits) - 1);
    u64 k = (top - 1) / two_n;
    while ((int)out.size() < count) {
        CK_CHECK(k > 0, CKKS_EINVAL, "ran out of NTT-friendly primes");
        u64 q = k * two_n + 1;
        if (q <= top && is_prime(q) && !exclude.count(q)) out.push_back(q);
        --k;
    }
    return out;
}

static u64 nearest_prime(double target, u64 two_n, const std::set<u64>& used) {
    long long k0 = (long long)floor((target - 1.0) / (double)two_n);
    u64 best = 0;
    double bestd = 0;
    for (int dir = 0; dir < 2; ++dir) {
        long long k = k0 + dir;
        long long step = dir == 0 ? -1 : 1;
        u64 q;
        for (;;) {
            CK_CHECK(k > 0, CKKS_EINVAL, "no NTT-friendly prime near the target scale");
            q = (u64)k * two_n + 1;
            if (is_prime(q) && !used.count(q)) break;
            k += step;
        }
        double d = fabs((double)q - target);
        if (best == 0 || d < bestd || (d == bestd && q < best)) {
            best = q;
            bestd = d;
        }
    }
    return best;
}

void build_chain(const ckks_params& P, std::vector<u64>& q, std::vector<u64>& p, std::vector<double>& delta) {
    const u64 two_n = 2ULL << P.log_n;
    const int nq = P.n_q, L = nq - 1;
    const int alpha = (nq + P.dnum - 1) / P.dnum;
    const int np = P.n_p > 0 ? P.n_p : alpha;
    std::set<u64> used;
    q.assign(nq, 0);
    delta.assign(nq, 0.0);
    q[0] = largest_primes(P.q0_bits, two_n, 1, used)[0];
    used.insert(q[0]);
    p = largest_primes(P.p_bits, two_n, np, used);
    for (u64 x : p) used.insert(x);
    const int c = L - P.n_boot;
    struct Seg {
        int top, bottom, bits;
    } segs[2] = {{L, c + 1, P.boot_bits}, {c, 1, P.scale_bits}};
    for (const Seg& sg : segs) {
        if (sg.top < sg.bottom) continue;
        const double base = ldexp(1.0, sg.bits);
        delta[sg.top] = base;
        for (int l = sg.top; l >= sg.bottom; --l) {
            const double target = (delta[l] * delta[l]) / base;
            const u64 ql = nearest_prime(target, two_n, used);
            used.insert(ql);
            q[l] = ql;
            if (l > sg.bottom || sg.bottom == 1) delta[l - 1] = (delta[l] * delta[l]) / (double)ql;
        }
    }
}

// smallest primitive 2N-th root of unity mod q
u64 smallest_root_2n(u64 q, int n) {
    CK_CHECK((q - 1) % (2ULL * n) == 0, CKKS_EINVAL, "prime is not 1 mod 2N");
    u64 c = 0;
    for (u64 x = 2;; ++x) {
        c = powmod(x, (q - 1) / (2ULL * n), q);
        if (powmod(c, (u64)n, q) == q - 1) break;
    }
    u64 best = c, c2 = mulmod(c, c, q), cur = c;
    for (int i = 0; i < n - 1; ++i) {
        cur = mulmod(cur, c2, q);
        if (cur < best) best = cur;
    }
    return best;
}

// cumulative table of the truncated discrete Gaussian: weight exp(-(v v) / (2 sigma^2)),
// v = -19..19; T[k] = floor(2^63 * cum_k / Z), last entry 2^63
void gauss_table(double sigma, u64* t) {
    double w[39], z = 0.0, cum = 0.0;
    for (int k = 0; k < 39; ++k) {
        int v = k - 19;
        w[k] = exp(-(double)(v * v) / (2.0 * sigma * sigma));
        z += w[k];
    }
    for (int k = 0; k < 39; ++k) {
        cum += w[k];
        t[k] = (u64)(cum / z * 9223372036854775808.0);
    }
    t[38] = 9223372036854775808ULL;
}
