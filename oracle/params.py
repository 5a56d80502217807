"""RNS-CKKS parameters of the oracle: NTT-friendly primes, roots, scale ladder.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper fixes N, L, dnum, Delta and h (Table 3) and defers the scheme itself to
RNS-CKKS (Sec. 2.1); it is silent on how the primes are chosen.  The reading
used here (identical rule on the CUDA side, implemented separately):

* q0 ("base prime"): the largest prime q < 2^q0_bits with q = 1 mod 2N.
* special primes p_0..p_{alpha-1}: the next largest such primes below
  2^p_bits, distinct from q0.
* scaling primes, chosen top-down so that every level keeps one canonical scale.
  The chain has two segments: "bootstrapping" levels c+1..L (CtoS and EvalMod,
  which need more precision than the message scale) and "circuit" levels 1..c
  at Delta = 2^scale_bits (Table 3).  Within a segment with base b:
  Delta_top = 2^b; going down, q_l is the unused prime = 1 mod 2N nearest to
  Delta_l^2 / 2^b and Delta_{l-1} = Delta_l^2 / q_l.  A product of two level-l
  ciphertexts (scale Delta_l each) rescaled by q_l then lands exactly on
  Delta_{l-1} (Sec. 2.4, "Rescaling").  The boot segment is chosen first.
* psi_i: the smallest primitive 2N-th root of unity mod q_i.
* digits: alpha = ceil((L+1)/dnum) consecutive Q-limbs per digit, alpha
  special primes.
"""
import math
from functools import lru_cache


def is_prime(n):
    """Deterministic Miller-Rabin for n < 3.3e24 (bases 2..37)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def primes_below(bits, two_n, count, exclude=()):
    """The `count` largest primes q < 2^bits with q = 1 mod two_n, skipping `exclude`."""
    out = []
    k = ((1 << bits) - 2) // two_n
    while len(out) < count:
        q = k * two_n + 1
        if q < (1 << bits) and is_prime(q) and q not in exclude:
            out.append(q)
        k -= 1
        if k <= 0:
            raise ValueError("ran out of NTT-friendly primes")
    return out


def nearest_prime(target, two_n, used):
    """Prime q = 1 mod two_n nearest to the real `target`, not in `used` (ties -> smaller)."""
    k0 = int(math.floor((target - 1.0) / two_n))
    best = None
    for direction in (0, 1):
        k = k0 + direction
        step = -1 if direction == 0 else 1
        while True:
            q = k * two_n + 1
            if q > 2 and is_prime(q) and q not in used:
                break
            k += step
        dist = abs(float(q) - target)
        if best is None or dist < best[0] or (dist == best[0] and q < best[1]):
            best = (dist, q)
    return best[1]


def smallest_primitive_root_2n(q, n):
    """Smallest psi in [2, q) with psi^N = -1 mod q (a primitive 2N-th root)."""
    assert (q - 1) % (2 * n) == 0
    x = 2
    while True:
        c = pow(x, (q - 1) // (2 * n), q)
        if pow(c, n, q) == q - 1:
            break
        x += 1
    # every primitive 2N-th root is c^k, k odd; take the smallest
    best = c
    c2 = c * c % q
    cur = c
    for _ in range(n - 1):
        cur = cur * c2 % q
        if cur < best:
            best = cur
    return best


class Params:
    """One RNS-CKKS parameter set.

    logn        log2 ring degree N
    n_q         number of Q-limbs (levels 0..L with L = n_q - 1)
    dnum        number of key-switching digits
    q0_bits, scale_bits, p_bits   bit sizes as in Table 3 / the configs
    h           Hamming weight of the secret (0 = uniform ternary)
    sigma       error standard deviation
    n_p         number of special primes (default alpha)
    boot_bits, n_boot   base and count of the top "bootstrapping" levels (0 = none)
    """

    def __init__(self, logn, n_q, dnum, q0_bits, scale_bits, p_bits, h=0, sigma=3.2,
                 n_p=None, boot_bits=0, n_boot=0):
        self.logn = logn
        self.n = 1 << logn
        self.n_q = n_q
        self.L = n_q - 1
        self.dnum = dnum
        self.alpha = -(-n_q // dnum)
        self.n_p = n_p or self.alpha
        self.boot_bits, self.n_boot = boot_bits, n_boot
        self.n_circuit = n_q - 1 - n_boot
        self.q0_bits, self.scale_bits, self.p_bits = q0_bits, scale_bits, p_bits
        self.h = h
        self.sigma = sigma
        self.q, self.p, self.delta = _chain(logn, n_q, self.n_p, q0_bits, scale_bits, p_bits,
                                            boot_bits, n_boot)
        self.psi_q = [smallest_primitive_root_2n(x, self.n) for x in self.q]
        self.psi_p = [smallest_primitive_root_2n(x, self.n) for x in self.p]

    # global prime ids: q_0..q_L are 0..L, p_j is L+1+j
    def prime_ids(self, level, with_p=False):
        ids = list(range(level + 1))
        if with_p:
            ids += [self.n_q + j for j in range(self.n_p)]
        return ids

    def moduli(self, level, with_p=False):
        return list(self.q[: level + 1]) + (list(self.p) if with_p else [])

    def psis(self, level, with_p=False):
        return list(self.psi_q[: level + 1]) + (list(self.psi_p) if with_p else [])

    def digits(self, level):
        """Digit d covers Q-limbs [d*alpha, min((d+1)*alpha, level+1))."""
        out = []
        for d in range(self.dnum):
            lo, hi = d * self.alpha, min((d + 1) * self.alpha, level + 1)
            if lo < hi:
                out.append(list(range(lo, hi)))
        return out


@lru_cache(maxsize=None)
def _chain(logn, n_q, n_p, q0_bits, scale_bits, p_bits, boot_bits=0, n_boot=0):
    two_n = 2 << logn
    q0 = primes_below(q0_bits, two_n, 1)[0]
    p = primes_below(p_bits, two_n, n_p, exclude={q0})
    used = {q0, *p}
    L = n_q - 1
    c = L - n_boot
    delta = [0.0] * n_q
    q = [0] * n_q
    q[0] = q0
    for top, bottom, bits in ((L, c + 1, boot_bits), (c, 1, scale_bits)):
        if top < bottom:
            continue
        base = float(2 ** bits)
        delta[top] = base
        for l in range(top, bottom - 1, -1):
            target = (delta[l] * delta[l]) / base
            ql = nearest_prime(target, two_n, used)
            used.add(ql)
            q[l] = ql
            if l > bottom or bottom == 1:
                delta[l - 1] = (delta[l] * delta[l]) / float(ql)
    return tuple(q), tuple(p), tuple(delta)


# --- named parameter sets -----------------------------------------------------
def cfg1_params():
    """N=2^12, 6 primes (q0 60-bit, 3 x 40-bit scaling, 2 x 60-bit special), dnum=2,
    scale 2^40, uniform ternary secret, sigma 3.2."""
    return Params(12, 4, 2, 60, 40, 60, h=0)


def cfg2_params():
    """N=2^16, 24 Q-limbs: q0 60-bit, 9 circuit levels at Delta=2^42 (Table 3), 14
    bootstrapping levels at 2^48; dnum=3 (8 limbs per digit) with 7 special 60-bit primes
    (P above the largest digit); Hamming weight 192 (Table 3); log PQ = 1530 <= 1555."""
    return Params(16, 24, 3, 60, 42, 60, h=192, n_p=7, boot_bits=48, n_boot=14)


# --- stream tags of the seeded randomness ---------------------------------------
# tag = kind << 56 | a << 16 | b ; the i-th word of a stream is SplitMix64 output i
# from state stream_key(seed, tag).
K_SK, K_SK_SIGN, K_PK_A, K_PK_E, K_SWK_A, K_SWK_E = 1, 2, 3, 4, 5, 6
K_ENC_U, K_ENC_E0, K_ENC_E1, K_ENCSK_A, K_ENCSK_E = 7, 8, 9, 10, 11


def tag(kind, a=0, b=0):
    return (kind << 56) | (a << 16) | b
