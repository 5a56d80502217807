// Device modular arithmetic for 64-bit RNS limbs (primes q < 2^61).
//
// mul_mod: Barrett reduction of the 128-bit product with s = bitlen(q),
//          mu = floor(2^(2s) / q): t = ((x >> (s-1)) * mu) >> (s+1) underestimates
//          floor(x/q) by at most 2, so r = x - t q lies in [0, 3q) and two
//          conditional subtractions finish it.
// mul_shoup: product with a constant w whose companion w' = floor(w 2^64 / q) is
//          precomputed (Shoup): r = a w - umulhi(a, w') q lies in [0, 2q).
#pragma once
#include <stdint.h>

typedef unsigned long long u64;

struct DevMod {
    u64 q;
    u64 mu;
    int s;
};

#ifdef __CUDACC__

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}

__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + (q - b); }

__device__ __forceinline__ u64 neg_mod(u64 a, u64 q) { return a ? q - a : 0; }

__device__ __forceinline__ u64 barrett_reduce128(u64 hi, u64 lo, const DevMod& m) {
    // requires (hi:lo) < 2^(2s)
    u64 x1 = (hi << (65 - m.s)) | (lo >> (m.s - 1));
    u64 tl = x1 * m.mu, th = __umul64hi(x1, m.mu);
    u64 t = (th << (63 - m.s)) | (tl >> (m.s + 1));
    u64 r = lo - t * m.q;
    if (r >= m.q) r -= m.q;
    if (r >= m.q) r -= m.q;
    return r;
}

__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const DevMod& m) {
    return barrett_reduce128(__umul64hi(a, b), a * b, m);
}

__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 wp, u64 q) {
    u64 hi = __umul64hi(a, wp);
    u64 r = a * w - hi * q;
    return r >= q ? r - q : r;
}

// (hi:lo) += x y, the 128-bit product formed from four 32 x 32 products in one carry chain of
// 32-bit multiply-adds (the low and high halves of the 64-bit product share their partial
// products)
__device__ __forceinline__ void mac128(u64& lo, u64& hi, u64 x, u64 y) {
    unsigned a0, a1, a2, a3;
    asm("mov.b64 {%0, %1}, %4;\n\t"
        "mov.b64 {%2, %3}, %5;"
        : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
        : "l"(lo), "l"(hi));
    const unsigned x0 = (unsigned)x, x1 = (unsigned)(x >> 32), y0 = (unsigned)y, y1 = (unsigned)(y >> 32);
    asm("mad.lo.cc.u32  %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.u32    %3, %5, %7, %3;\n\t"
        "mad.lo.cc.u32  %1, %4, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
        "addc.u32       %3, %3, 0;\n\t"
        "mad.lo.cc.u32  %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "addc.u32       %3, %3, 0;"
        : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3)
        : "r"(x0), "r"(x1), "r"(y0), "r"(y1));
    asm("mov.b64 %0, {%2, %3};\n\t"
        "mov.b64 %1, {%4, %5};"
        : "=l"(lo), "=l"(hi)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3));
}

// reduce an arbitrary 64-bit word mod q (q < 2^61): (0:x) < 2^64 <= 2^(2s) whenever s >= 32
__device__ __forceinline__ u64 reduce64(u64 x, const DevMod& m) { return barrett_reduce128(0, x, m); }

// centred residue of v mod qs, reduced mod qt
__device__ __forceinline__ u64 centred_to(u64 v, u64 qs, const DevMod& t) {
    if (v <= (qs >> 1)) return v >= t.q ? reduce64(v, t) : v;
    u64 d = qs - v;  // |v - qs|
    d = d >= t.q ? reduce64(d, t) : d;
    return d ? t.q - d : 0;
}

__device__ __forceinline__ unsigned brev_bits(unsigned x, int bits) { return __brev(x) >> (32 - bits); }

// index of the NTT slot holding a(X^g) at slot i (bit-reversed evaluation order):
// slot i is the evaluation at psi^(2 rev(i) + 1); a(X^g) there is a at psi^((2 rev(i)+1) g)
__device__ __forceinline__ unsigned galois_src(unsigned i, u64 g, int logn) {
    unsigned r = brev_bits(i, logn);
    u64 e = ((2ull * r + 1ull) * g) & ((2ull << logn) - 1ull);
    return brev_bits((unsigned)((e - 1) >> 1), logn);
}
#endif  // __CUDACC__
