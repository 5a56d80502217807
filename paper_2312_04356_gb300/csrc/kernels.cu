// Device kernels of the RNS-CKKS hot path and their launchers.
//
// Layout: a polynomial is [limb][N] uint64, limb k of an array of several
// polynomials uses the prime with global id ids[k % lpp].  One CTA row of the
// grid (blockIdx.y) is one limb, so the modulus is uniform inside a CTA.
#include "launch.cuh"

#include <atomic>

#include <cooperative_groups.h>
namespace cg = cooperative_groups;

// ------------------------------------------------------------ DevBuf -------
thread_local const DevAlloc* tl_alloc = nullptr;

DevBuf::DevBuf(size_t w, cudaStream_t s) : words(w), stream(s) {
    if (w && tl_alloc && tl_alloc->alloc) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CUDA_CHECK(cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusNone) {
            void* p = tl_alloc->alloc(tl_alloc->user, w * sizeof(u64), (void*)s);
            CK_CHECK(p != nullptr, CKKS_ENOMEM, "the caller's device allocator returned NULL");
            CK_CHECK(((uintptr_t)p & 15) == 0, CKKS_EINVAL, "the caller's device allocator returned a pointer "
                                                            "that is not 16-byte aligned");
            ptr = (u64*)p;
            al = *tl_alloc;
            return;
        }
    }
    if (w) {
        cudaError_t e = cudaMallocAsync((void**)&ptr, w * sizeof(u64), s);
        if (e != cudaSuccess) {
            ptr = nullptr;
            CK_THROW(CKKS_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
        }
    }
}
DevBuf::~DevBuf() { reset(); }
DevBuf& DevBuf::operator=(DevBuf&& o) noexcept {
    if (this != &o) {
        reset();
        ptr = o.ptr;
        words = o.words;
        stream = o.stream;
        al = o.al;
        o.ptr = nullptr;
        o.words = 0;
        o.al = DevAlloc();
    }
    return *this;
}
void DevBuf::reset() {
    if (ptr) {
        if (al.free)
            al.free(al.user, ptr, words * sizeof(u64), (void*)stream);
        else if (!al.alloc)
            cudaFreeAsync(ptr, stream);
    }
    ptr = nullptr;
    words = 0;
    al = DevAlloc();
}

static cudaEvent_t take_event(const ckks_ctx* c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

KTimer::KTimer(const ckks_ctx* ctx, const char* nm, double algo_bytes) : c(ctx), name(nm), bytes(algo_bytes) {
    ++c->launches;
    if (c->timing) {
        a = take_event(c);
        b = take_event(c);
        cudaEventRecord(a, c->stream);
    }
}

KTimer::~KTimer() {
    if (a) {
        cudaEventRecord(b, c->stream);
        c->pending.push_back({name, a, b, bytes});
        if (c->pending.size() > 4096) c->collect_timing();
    }
}

void ckks_ctx::collect_timing() const {
    if (pending.empty()) return;
    cudaEventSynchronize(pending.back().b);
    for (const Pending& p : pending) {
        float ms = 0;
        cudaEventElapsedTime(&ms, p.a, p.b);
        KStat& st = kstats[p.name];
        st.launches += 1;
        st.ms += ms;
        st.bytes += p.bytes;
        event_pool.push_back(p.a);
        event_pool.push_back(p.b);
    }
    pending.clear();
}

namespace {

constexpr int EW_THREADS = 256;

inline dim3 ew_grid(int n, int nlimbs) {
    int x = n / (EW_THREADS * 4);
    if (x < 1) x = 1;
    return dim3(x, nlimbs);
}

#define EW_LOOP(n) for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < (n); j += gridDim.x * blockDim.x)

// grid of the one-thread-per-V-words kernels
inline dim3 ewv_grid(int n, int nlimbs, int v) {
    int x = n / (EW_THREADS * v);
    if (x < 1) x = 1;
    return dim3(x, nlimbs);
}
inline bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }
// words per thread of the elementwise kernels when every pointer is 16-byte aligned
constexpr int EWV_VEC = 4;
#define EWV_LAUNCH(K, vec, nl, ...)                                                          \
    do {                                                                                     \
        if (vec)                                                                             \
            klaunch(c, K<EWV_VEC>, ewv_grid(c->n, (nl), EWV_VEC), EW_THREADS, 0, __VA_ARGS__); \
        else                                                                                 \
            klaunch(c, K<1>, ewv_grid(c->n, (nl), 1), EW_THREADS, 0, __VA_ARGS__);        \
    } while (0)

// ------------------------------------------------------------------ NTT ----
// One pass covers `c` consecutive butterfly stages s0..s0+c-1 (stage s: 2^s groups,
// stride t = N >> (s+1)).  Over those stages only index bits log2(T1)..log2(T0) move
// (T0 = N >> (s0+1), T1 = N >> (s0+c)), so the limb splits into independent
// sub-problems of 2^c elements j = hi*2T0 + k*T1 + lo.  A CTA stages SUB of them
// (4096 elements) in shared memory, runs the c stages, and writes them back.
constexpr int NTT_THREADS = 256;

template <bool INV>
__global__ void __launch_bounds__(NTT_THREADS)
    k_ntt_pass(u64* __restrict__ data, const DevPrime* __restrict__ primes, const int* __restrict__ ids, int lpp,
               size_t pstride, int logn, int s0, int c, int logsub, int scale_out, const u64* __restrict__ osc) {
    griddep_entry();
    extern __shared__ u64 sm[];
    const int limb = blockIdx.y;
    const DevPrime* P = primes + ids[limb % lpp];
    const u64 q = P->m.q;
    u64* a = data + (size_t)(limb / lpp) * pstride + ((size_t)(limb % lpp) << logn);
    const int span = 1 << c;
    const int SUB = 1 << logsub;
    const int stride = SUB > 1 ? SUB + 1 : 1;
    const int logT1 = logn - s0 - c;
    const int T1 = 1 << logT1;
    const int log2T0 = logn - s0;
    const int sid0 = blockIdx.x * SUB;
    const int total = SUB << c;

    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int s, k;
        if (T1 == 1) {
            s = e >> c;
            k = e & (span - 1);
        } else {
            k = e >> logsub;
            s = e & (SUB - 1);
        }
        int sid = sid0 + s;
        size_t j = ((size_t)(sid >> logT1) << log2T0) + ((size_t)k << logT1) + (sid & (T1 - 1));
        sm[k * stride + s] = a[j];
    }
    __syncthreads();

    const int nbf = total >> 1;
    for (int u = 0; u < c; ++u) {
        const int uu = INV ? (c - 1 - u) : u;
        const int sg = s0 + uu;               // global stage
        const int lt = c - 1 - uu;            // log2 of the local stride
        const int tk = 1 << lt;
        for (int e = threadIdx.x; e < nbf; e += blockDim.x) {
            const int s = e & (SUB - 1);
            const int b = e >> logsub;
            const int k = ((b >> lt) << (lt + 1)) | (b & (tk - 1));
            const int sid = sid0 + s;
            const size_t j = ((size_t)(sid >> logT1) << log2T0) + ((size_t)k << logT1) + (sid & (T1 - 1));
            const int widx = (1 << sg) + (int)(j >> (logn - sg));
            u64* px = sm + k * stride + s;
            u64* py = sm + (k + tk) * stride + s;
            const u64 x = *px, y = *py;
            if (!INV) {
                const ulonglong2 w = P->tw[widx];
                const u64 v = mul_shoup(y, w.x, w.y, q);
                *px = add_mod(x, v, q);
                *py = sub_mod(x, v, q);
            } else {
                *px = add_mod(x, y, q);
                const ulonglong2 w = P->itw[widx];
                *py = mul_shoup(sub_mod(x, y, q), w.x, w.y, q);
            }
        }
        __syncthreads();
    }

    // the inverse transform's final factor: N^{-1}, or per row a caller-given (w, w') Shoup pair
    const u64 ninv = osc ? osc[2 * (limb % lpp)] : P->n_inv, ninvp = osc ? osc[2 * (limb % lpp) + 1] : P->n_inv_p;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int s, k;
        if (T1 == 1) {
            s = e >> c;
            k = e & (span - 1);
        } else {
            k = e >> logsub;
            s = e & (SUB - 1);
        }
        int sid = sid0 + s;
        size_t j = ((size_t)(sid >> logT1) << log2T0) + ((size_t)k << logT1) + (sid & (T1 - 1));
        u64 v = sm[k * stride + s];
        if (scale_out) v = mul_shoup(v, ninv, ninvp, q);
        a[j] = v;
    }
}

// ---- fast path for N = 2^16: two passes of 8 stages, each as two radix-16 rounds ----
// A pass works on 256-element sub-problems (k = 0..255), 16 threads per sub-problem,
// 16 values per thread in registers.  Round A covers local stages u = 0..3 on the
// elements k = t + 16 i, round B covers u = 4..7 on k = 16 t + i; one shared-memory
// exchange separates them.  Butterflies are Harvey's lazy forms: forward values stay in
// [0, 4q), inverse values in [0, 2q); the last forward pass and the N^{-1} scaling
// return canonical residues.  Twiddle of local stage u for element k of sub-problem hi:
// index 2^(s0+u) + hi 2^u + (k >> (8 - u)).
constexpr int F_STRIDE = 273;             // shared words per sub-problem: 256 + 16 pad, odd
__device__ __forceinline__ int f_slot(int sp, int k) { return sp * F_STRIDE + k + (k >> 4); }

// Forward butterflies reduce the upper input only on odd local stages (threshold 4q): an
// uncorrected stage maps inputs in [0, b q) to [0, (b + 2) q), a corrected one (valid for
// b <= 8) to [0, 6q).  From canonical inputs the values stay below 8q, which fits in 64
// bits for every prime below 2^61; each pass ends in [0, 6q).
template <bool CORR>
__device__ __forceinline__ void ct_bfly(u64& x, u64& y, u64 w, u64 wp, u64 q, u64 q2, u64 q4) {
    if (CORR && x >= q4) x -= q4;
    const u64 t = y * w - __umul64hi(y, wp) * q;   // [0, 2q)
    y = x - t + q2;
    x = x + t;
}
__device__ __forceinline__ void gs_bfly(u64& x, u64& y, u64 w, u64 wp, u64 q, u64 q2) {
    u64 s = x + y;
    if (s >= q2) s -= q2;
    const u64 d = x - y + q2;
    y = d * w - __umul64hi(d, wp) * q;             // [0, 2q)
    x = s;
}

// forward round over 4 local stages u0..u0+3; element i of the thread has index k(i);
// tw index offset for lower element i at stage u: base_u + (k(i) >> (8 - u))
template <bool ROUND_B>
__device__ __forceinline__ void fwd_round(u64 (&x)[16], int t, int hi, int s0, const DevPrime* __restrict__ P,
                                          u64 q, u64 q2) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int u = (ROUND_B ? 4 : 0) + s;
        const int is = 8 >> s;
        const int base = (1 << (s0 + u)) + (hi << u);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (i & is) continue;
            const int idx = ROUND_B ? base + (t << s) + (i >> (4 - s)) : base + (i >> (4 - s));
            const ulonglong2 w = __ldg(P->tw + idx);
            if (u & 1)
                ct_bfly<true>(x[i], x[i + is], w.x, w.y, q, q2, 2 * q2);
            else
                ct_bfly<false>(x[i], x[i + is], w.x, w.y, q, q2, 2 * q2);
        }
    }
}

template <bool ROUND_B>
__device__ __forceinline__ void inv_round(u64 (&x)[16], int t, int hi, int s0, const DevPrime* __restrict__ P,
                                          u64 q, u64 q2) {
#pragma unroll
    for (int s = 3; s >= 0; --s) {
        const int u = (ROUND_B ? 4 : 0) + s;
        const int is = 8 >> s;
        const int base = (1 << (s0 + u)) + (hi << u);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (i & is) continue;
            const int idx = ROUND_B ? base + (t << s) + (i >> (4 - s)) : base + (i >> (4 - s));
            const ulonglong2 w = __ldg(P->itw + idx);
            gs_bfly(x[i], x[i + is], w.x, w.y, q, q2);
        }
    }
}

// Input of the inverse transform's first pass when it is not the data array itself (SRC
// kernels): row k reads src + (k / lpp) * src_pstride + (k % lpp) N and the result goes to the
// data array, so the input is left as it is (no copy before an out-of-place transform).
// ow != 0 replaces the final factor N^{-1} by the Shoup pair (ow, owp), e.g. k N^{-1} to
// multiply the result by the integer k.
struct NttSrc {
    const u64* src;
    size_t src_pstride;
    u64 ow, owp;
};

// COL: sub-problems are columns (s0 = 0, T1 = 256, element j = k*256 + lo), threads with
//      consecutive tid take consecutive columns.  ROW: sub-problems are contiguous rows
//      (s0 = 8, T1 = 1, j = hi*256 + k), consecutive tid take consecutive k.
template <bool COL, bool INV, int SUBS, int MINB, bool SRC = false>
__global__ void __launch_bounds__(16 * SUBS, MINB) k_ntt16(u64* __restrict__ data, const DevPrime* __restrict__ primes,
                                                    const int* __restrict__ ids, int lpp, size_t pstride,
                                                    const int* __restrict__ loff, const u64* __restrict__ osc,
                                                    NttSrc io) {
    static_assert(!SRC || (INV && !COL), "only the inverse transform's first pass reads a separate source");
    griddep_entry();
    __shared__ u64 sm[SUBS * F_STRIDE];
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const DevPrime* P = primes + ids[r];
    const u64 q = P->m.q, q2 = 2 * q;
    u64* a = data + (size_t)(limb / lpp) * pstride + ((size_t)(loff ? loff[r] : r) << 16);
    const int tid = threadIdx.x;
    const int sp = COL ? (tid % SUBS) : (tid >> 4);
    const int t = COL ? (tid / SUBS) : (tid & 15);
    const int sub = blockIdx.x * SUBS + sp;            // global sub-problem: column lo or row hi
    const int s0 = COL ? 0 : 8;
    const int hi = COL ? 0 : sub;
    u64 x[16];
    auto gidx = [&](int k) -> size_t { return COL ? ((size_t)k << 8) + sub : ((size_t)sub << 8) + k; };

    if (!INV) {
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = a[gidx(t + 16 * i)];
        fwd_round<false>(x, t, hi, s0, P, q, q2);
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[f_slot(sp, t + 16 * i)] = x[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = sm[f_slot(sp, 16 * t + i)];
        fwd_round<true>(x, t, hi, s0, P, q, q2);
        if (COL) {
#pragma unroll
            for (int i = 0; i < 16; ++i) a[gidx(16 * t + i)] = x[i];     // lazy, [0, 6q)
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                u64 v = x[i];
                if (v >= 2 * q2) v -= 2 * q2;
                if (v >= q2) v -= q2;
                if (v >= q) v -= q;
                x[i] = v;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 16; ++i) sm[f_slot(sp, 16 * t + i)] = x[i];
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 16; ++i) a[gidx(t + 16 * i)] = sm[f_slot(sp, t + 16 * i)];
        }
    } else {
        if (COL) {
#pragma unroll
            for (int i = 0; i < 16; ++i) x[i] = a[gidx(16 * t + i)];
        } else {
            const u64* sr = SRC ? io.src + (size_t)(limb / lpp) * io.src_pstride + ((size_t)r << 16) : a;
#pragma unroll
            for (int i = 0; i < 16; ++i) sm[f_slot(sp, t + 16 * i)] = sr[gidx(t + 16 * i)];
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 16; ++i) x[i] = sm[f_slot(sp, 16 * t + i)];
            __syncthreads();
        }
        inv_round<true>(x, t, hi, s0, P, q, q2);
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[f_slot(sp, 16 * t + i)] = x[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = sm[f_slot(sp, t + 16 * i)];
        inv_round<false>(x, t, hi, s0, P, q, q2);
        if (COL) {
            const u64 ni = io.ow ? io.ow : osc ? osc[2 * r] : P->n_inv;
            const u64 nip = io.ow ? io.owp : osc ? osc[2 * r + 1] : P->n_inv_p;
#pragma unroll
            for (int i = 0; i < 16; ++i) a[gidx(t + 16 * i)] = mul_shoup(x[i], ni, nip, q);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) a[gidx(t + 16 * i)] = x[i];     // lazy, [0, 2q)
        }
    }
}

// ---- the same pass with 4 values per thread: four radix-4 register rounds (local stages
// 2r, 2r+1), three shared-memory exchanges, 64 threads per sub-problem and 4 sub-problems
// per 256-thread CTA: four times the threads of k_ntt16, for launches over few limbs.
// In round r thread t holds k0 + {0, e, d, d + e} (d = 128 >> 2r, e = d / 2), k0 = t with
// zero bits inserted at the positions of d and e.  Butterflies, twiddle indices and the
// lazy bounds are those of k_ntt16, so both kernels return the same residues.
__device__ __forceinline__ int ins0(int t, int p) { return ((t >> p) << (p + 1)) | (t & ((1 << p) - 1)); }

template <bool COL, bool INV, bool SRC = false>
__global__ void __launch_bounds__(256) k_ntt16s(u64* __restrict__ data, const DevPrime* __restrict__ primes,
                                                const int* __restrict__ ids, int lpp, size_t pstride,
                                                const int* __restrict__ loff, const u64* __restrict__ osc,
                                                NttSrc io) {
    static_assert(!SRC || (INV && !COL), "only the inverse transform's first pass reads a separate source");
    griddep_entry();
    __shared__ u64 sm[4 * F_STRIDE];
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const DevPrime* P = primes + ids[r];
    const u64 q = P->m.q, q2 = 2 * q;
    u64* a = data + (size_t)(limb / lpp) * pstride + ((size_t)(loff ? loff[r] : r) << 16);
    const int tid = threadIdx.x;
    const int sp = COL ? (tid & 3) : (tid >> 6);
    const int t = COL ? (tid >> 2) : (tid & 63);
    const int sub = blockIdx.x * 4 + sp;
    const int s0 = COL ? 0 : 8;
    const int hi = COL ? 0 : sub;
    auto gidx = [&](int k) -> size_t { return COL ? ((size_t)k << 8) + sub : ((size_t)sub << 8) + k; };
    u64 x[4];
    int k0 = 0;
    if (!INV) {
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int u = 2 * rr, d = 128 >> u, e = d >> 1;
            k0 = ins0(ins0(t, 6 - u), 7 - u);
            const int ks[4] = {k0, k0 + e, k0 + d, k0 + d + e};
            if (rr == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) x[i] = a[gidx(ks[i])];
            } else {
                __syncthreads();
#pragma unroll
                for (int i = 0; i < 4; ++i) x[i] = sm[f_slot(sp, ks[i])];
            }
            // stage u (odd/even correction as in k_ntt16): pairs (0, 2), (1, 3), one twiddle
            {
                const ulonglong2 w = __ldg(P->tw + (1 << (s0 + u)) + (hi << u) + (k0 >> (8 - u)));
                ct_bfly<false>(x[0], x[2], w.x, w.y, q, q2, 2 * q2);
                ct_bfly<false>(x[1], x[3], w.x, w.y, q, q2, 2 * q2);
            }
            // stage u + 1 (odd): pairs (0, 1), (2, 3)
            {
                const int base = (1 << (s0 + u + 1)) + (hi << (u + 1));
                const ulonglong2 w0 = __ldg(P->tw + base + (k0 >> (7 - u)));
                const ulonglong2 w1 = __ldg(P->tw + base + ((k0 + d) >> (7 - u)));
                ct_bfly<true>(x[0], x[1], w0.x, w0.y, q, q2, 2 * q2);
                ct_bfly<true>(x[2], x[3], w1.x, w1.y, q, q2, 2 * q2);
            }
            if (rr < 3) {
                __syncthreads();
#pragma unroll
                for (int i = 0; i < 4; ++i) sm[f_slot(sp, ks[i])] = x[i];
            } else if (COL) {
#pragma unroll
                for (int i = 0; i < 4; ++i) a[gidx(ks[i])] = x[i];     // lazy, [0, 6q)
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    u64 v = x[i];
                    if (v >= 2 * q2) v -= 2 * q2;
                    if (v >= q2) v -= q2;
                    if (v >= q) v -= q;
                    a[gidx(ks[i])] = v;
                }
            }
        }
    } else {
#pragma unroll
        for (int rr = 3; rr >= 0; --rr) {
            const int u = 2 * rr, d = 128 >> u, e = d >> 1;
            k0 = ins0(ins0(t, 6 - u), 7 - u);
            const int ks[4] = {k0, k0 + e, k0 + d, k0 + d + e};
            if (rr == 3) {
                const u64* sr = SRC ? io.src + (size_t)(limb / lpp) * io.src_pstride + ((size_t)r << 16) : a;
#pragma unroll
                for (int i = 0; i < 4; ++i) x[i] = sr[gidx(ks[i])];
            } else {
                __syncthreads();
#pragma unroll
                for (int i = 0; i < 4; ++i) x[i] = sm[f_slot(sp, ks[i])];
            }
            // stage u + 1 first: pairs (0, 1), (2, 3)
            {
                const int base = (1 << (s0 + u + 1)) + (hi << (u + 1));
                const ulonglong2 w0 = __ldg(P->itw + base + (k0 >> (7 - u)));
                const ulonglong2 w1 = __ldg(P->itw + base + ((k0 + d) >> (7 - u)));
                gs_bfly(x[0], x[1], w0.x, w0.y, q, q2);
                gs_bfly(x[2], x[3], w1.x, w1.y, q, q2);
            }
            // stage u: pairs (0, 2), (1, 3)
            {
                const ulonglong2 w = __ldg(P->itw + (1 << (s0 + u)) + (hi << u) + (k0 >> (8 - u)));
                gs_bfly(x[0], x[2], w.x, w.y, q, q2);
                gs_bfly(x[1], x[3], w.x, w.y, q, q2);
            }
            if (rr > 0) {
                __syncthreads();
#pragma unroll
                for (int i = 0; i < 4; ++i) sm[f_slot(sp, ks[i])] = x[i];
            } else if (COL) {
                const u64 ni = io.ow ? io.ow : osc ? osc[2 * r] : P->n_inv;
                const u64 nip = io.ow ? io.owp : osc ? osc[2 * r + 1] : P->n_inv_p;
#pragma unroll
                for (int i = 0; i < 4; ++i) a[gidx(ks[i])] = mul_shoup(x[i], ni, nip, q);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) a[gidx(ks[i])] = x[i];     // lazy, [0, 2q)
            }
        }
    }
}

// ---- the whole N = 2^16 transform in one launch: a cluster of 8 CTAs per limb (512 threads
// each, 16 values per thread).  Forward: CTA r runs stages 0-7 on columns 32r .. 32r+31 (the
// COL pass of k_ntt16 with 32 sub-problems), writes them to its shared memory as [row][32],
// and after a cluster barrier reads rows 32r .. 32r+31 from all eight CTAs through
// distributed shared memory for stages 8-15 (the ROW pass).  Inverse: the same in reverse
// order.  Butterflies, twiddles and lazy bounds are those of k_ntt16, so the residues are
// identical; the data makes one trip through HBM instead of two.  Every thread of every CTA
// reaches both cluster barriers (no early exit), and the second barrier keeps each CTA's
// shared memory alive until the other CTAs have read it.
constexpr int CL_SUBS = 32, CL_THREADS = 512, CL_SMEM_WORDS = CL_SUBS * F_STRIDE;

template <bool INV>
__global__ void __cluster_dims__(8, 1, 1) __launch_bounds__(CL_THREADS, 2)
    k_ntt_cl(u64* __restrict__ data, const DevPrime* __restrict__ primes, const int* __restrict__ ids, int lpp,
             size_t pstride, const int* __restrict__ loff, const u64* __restrict__ osc, NttSrc io) {
    griddep_entry();
    extern __shared__ u64 sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const DevPrime* P = primes + ids[r];
    const u64 q = P->m.q, q2 = 2 * q;
    u64* a = data + (size_t)(limb / lpp) * pstride + ((size_t)(loff ? loff[r] : r) << 16);
    const int tid = threadIdx.x;
    // COL mapping: column 32 rank + spc, elements (rows) t + 16 i / 16 t + i
    const int spc = tid % CL_SUBS, tc = tid / CL_SUBS, col = CL_SUBS * rank + spc;
    // ROW mapping: row 32 rank + spr, elements (columns) t + 16 i / 16 t + i
    const int spr = tid >> 4, tr = tid & 15, row = CL_SUBS * rank + spr;
    u64 x[16];
    if (!INV) {
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = a[((size_t)(tc + 16 * i) << 8) + col];
        fwd_round<false>(x, tc, 0, 0, P, q, q2);
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[f_slot(spc, tc + 16 * i)] = x[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = sm[f_slot(spc, 16 * tc + i)];
        fwd_round<true>(x, tc, 0, 0, P, q, q2);                      // column col, rows 16 tc + i
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[(16 * tc + i) * CL_SUBS + spc] = x[i];
        cl.sync();
#pragma unroll
        for (int i = 0; i < 16; ++i) {                               // column tr + 16 i of row `row`
            const u64* src = cl.map_shared_rank(sm, i >> 1);
            x[i] = src[row * CL_SUBS + tr + 16 * (i & 1)];
        }
        cl.sync();
        fwd_round<false>(x, tr, row, 8, P, q, q2);
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[f_slot(spr, tr + 16 * i)] = x[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = sm[f_slot(spr, 16 * tr + i)];
        fwd_round<true>(x, tr, row, 8, P, q, q2);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            u64 v = x[i];
            if (v >= 2 * q2) v -= 2 * q2;
            if (v >= q2) v -= q2;
            if (v >= q) v -= q;
            x[i] = v;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[f_slot(spr, 16 * tr + i)] = x[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) a[((size_t)row << 8) + tr + 16 * i] = sm[f_slot(spr, tr + 16 * i)];
    } else {
        const u64* sr = io.src ? io.src + (size_t)(limb / lpp) * io.src_pstride + ((size_t)r << 16) : a;
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[f_slot(spr, tr + 16 * i)] = sr[((size_t)row << 8) + tr + 16 * i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = sm[f_slot(spr, 16 * tr + i)];
        __syncthreads();
        inv_round<true>(x, tr, row, 8, P, q, q2);
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[f_slot(spr, 16 * tr + i)] = x[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = sm[f_slot(spr, tr + 16 * i)];
        inv_round<false>(x, tr, row, 8, P, q, q2);                   // row `row`, columns tr + 16 i
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[spr * 256 + tr + 16 * i] = x[i];
        cl.sync();
        {
            const u64* src = cl.map_shared_rank(sm, tc >> 1);          // rows 16 tc + i live there
#pragma unroll
            for (int i = 0; i < 16; ++i) x[i] = src[(16 * (tc & 1) + i) * 256 + col];
        }
        cl.sync();
        inv_round<true>(x, tc, 0, 0, P, q, q2);
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[f_slot(spc, 16 * tc + i)] = x[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = sm[f_slot(spc, tc + 16 * i)];
        inv_round<false>(x, tc, 0, 0, P, q, q2);
        const u64 ni = io.ow ? io.ow : osc ? osc[2 * r] : P->n_inv;
        const u64 nip = io.ow ? io.owp : osc ? osc[2 * r + 1] : P->n_inv_p;
#pragma unroll
        for (int i = 0; i < 16; ++i) a[((size_t)(tc + 16 * i) << 8) + col] = mul_shoup(x[i], ni, nip, q);
    }
}

// few limbs: 64-thread CTAs (4 sub-problems) so that the grid still covers the SMs
// Variants (identical results): CTA of 16 or 4 sub-problems, register budget for 3 or 4
// resident 256-thread CTAs per SM.  ckks_autotune times them per limb-count class; the
// default (no tuning) is 16 sub-problems at >= 16 limbs, else 4, 80 registers.
enum NttVariant {
    NTT_V16_R80 = 0, NTT_V16_R64 = 1, NTT_V4_R80 = 2, NTT_V4_R64 = 3, NTT_X4 = 4, NTT_CL = 5, NTT_NVARIANTS = 6
};

template <bool COL, bool INV, bool SRC = false>
void launch_ntt16_variant(const ckks_ctx* cx, int v, u64* data, int nlimbs, const int* ids, int lpp,
                          size_t pstride, const int* loff, const u64* osc, const NttSrc& io) {
    switch (v) {
        case NTT_V16_R80:
            klaunch(cx, k_ntt16<COL, INV, 16, 3, SRC>, dim3(256 / 16, nlimbs), 256, 0,
                    data, cx->d_primes, ids, lpp, pstride, loff, osc, io);
            break;
        case NTT_V16_R64:
            klaunch(cx, k_ntt16<COL, INV, 16, 4, SRC>, dim3(256 / 16, nlimbs), 256, 0,
                    data, cx->d_primes, ids, lpp, pstride, loff, osc, io);
            break;
        case NTT_V4_R80:
            klaunch(cx, k_ntt16<COL, INV, 4, 8, SRC>, dim3(256 / 4, nlimbs), 64, 0,
                    data, cx->d_primes, ids, lpp, pstride, loff, osc, io);
            break;
        case NTT_V4_R64:
            klaunch(cx, k_ntt16<COL, INV, 4, 12, SRC>, dim3(256 / 4, nlimbs), 64, 0,
                    data, cx->d_primes, ids, lpp, pstride, loff, osc, io);
            break;
        default:
            klaunch(cx, k_ntt16s<COL, INV, SRC>, dim3(256 / 4, nlimbs), 256, 0,
                    data, cx->d_primes, ids, lpp, pstride, loff, osc, io);
            break;
    }
}

inline int ntt_class(int nlimbs) {
    int c = 0;
    while (c < 7 && (2 << c) <= nlimbs) ++c;   // classes: 1, 2-3, 4-7, 8-15, 16-31, 32-63, 64-127, >=128
    return c;
}

template <bool INV>
void launch_ntt_cl(const ckks_ctx* cx, u64* data, int nlimbs, const int* ids, int lpp, size_t pstride,
                   const int* loff, const u64* osc, const NttSrc& io) {
    static std::atomic<unsigned> done{0};
    allow_dynamic_smem((const void*)k_ntt_cl<INV>, CL_SMEM_WORDS * (int)sizeof(u64), done);
    klaunch(cx, k_ntt_cl<INV>, dim3(8, nlimbs), CL_THREADS, CL_SMEM_WORDS * sizeof(u64),
            data, cx->d_primes, ids, lpp, pstride, loff, osc, io);
}

// One whole N = 2^16 transform with variant v: the cluster kernel, or the two passes (forward:
// COL then ROW; inverse: ROW then COL).  Algorithmic bytes: one read and one write of the
// limbs per transform, split evenly over the two passes.
// (io: a separate source of the inverse's first pass and an output factor, as NttSrc
// describes)
template <bool INV>
void launch_ntt_variant(const ckks_ctx* cx, int v, u64* data, int nlimbs, const int* ids, int lpp, size_t pstride,
                        const int* loff, const u64* osc = nullptr, const NttSrc& io = NttSrc{}) {
    const char* nm = INV ? "ntt_inv" : "ntt_fwd";
    const double bytes = 2.0 * nlimbs * cx->n * 8.0;
    CK_CHECK(INV || !io.src, CKKS_EINVAL, "only the inverse transform reads a separate source");
    if (v == NTT_CL) {
        KTimer kt_(cx, nm, bytes);
        launch_ntt_cl<INV>(cx, data, nlimbs, ids, lpp, pstride, loff, osc, io);
        return;
    }
    {
        KTimer kt_(cx, nm, bytes / 2);
        if (INV && io.src)     // the inverse's first pass is the ROW pass
            launch_ntt16_variant<false, true, true>(cx, v, data, nlimbs, ids, lpp, pstride, loff, osc, io);
        else
            launch_ntt16_variant<!INV, INV>(cx, v, data, nlimbs, ids, lpp, pstride, loff, osc, io);
    }
    {
        KTimer kt_(cx, nm, bytes / 2);
        launch_ntt16_variant<INV, INV>(cx, v, data, nlimbs, ids, lpp, pstride, loff, osc, io);
    }
}

// the variant that transforms of nlimbs limbs use: the tuned one of their size class, else
// 16 sub-problems per CTA from 16 limbs on and 4 below
inline int ntt_pick(const ckks_ctx* cx, int nlimbs) {
    const int v = cx->ntt_choice[ntt_class(nlimbs)];
    return v >= 0 ? v : nlimbs >= 16 ? NTT_V16_R80 : NTT_V4_R80;
}

template <bool INV>
void launch_ntt_transform(const ckks_ctx* cx, u64* data, int nlimbs, const int* ids, int lpp, size_t pstride,
                          const int* loff = nullptr, const u64* osc = nullptr, const NttSrc& io = NttSrc{}) {
    launch_ntt_variant<INV>(cx, ntt_pick(cx, nlimbs), data, nlimbs, ids, lpp, pstride, loff, osc, io);
}

struct PassPlan {
    int s0, c;
};

inline std::vector<PassPlan> ntt_passes(int logn) {
    if (logn <= 12) return {{0, logn}};
    return {{0, logn - 8}, {logn - 8, 8}};
}

template <bool INV>
void launch_pass(const ckks_ctx* cx, u64* data, int nlimbs, const int* ids, int lpp, size_t pstride, PassPlan p,
                 int scale_out, const u64* osc = nullptr) {
    const int logn = cx->logn;
    int logsub = 12 - p.c;
    if (logsub < 0) logsub = 0;
    if (logsub > logn - p.c) logsub = logn - p.c;
    const int SUB = 1 << logsub;
    const int tiles = (1 << (logn - p.c)) / SUB;
    const int stride = SUB > 1 ? SUB + 1 : 1;
    const size_t smem = (size_t)stride * (1 << p.c) * sizeof(u64);
    dim3 grid(tiles, nlimbs);
    { KTimer kt_(cx, INV ? "ntt_inv" : "ntt_fwd", 2.0 * nlimbs * cx->n * 8.0 * p.c / logn);
    klaunch(cx, k_ntt_pass<INV>, grid, NTT_THREADS, smem, data, cx->d_primes, ids, lpp, pstride, logn, p.s0, p.c,
            logsub, scale_out, osc);
    }
}

// ----------------------------------------------------------- elementwise ----
// One thread per V consecutive words of a limb (V = 2 or 4: 16-byte loads and stores, used
// when every pointer of the launch is 16-byte aligned); all operands are loaded before any
// store, so in-place calls (o == a) are safe.
template <int V>
__device__ __forceinline__ void ldv(const u64* p, u64 (&r)[V]) {
    if constexpr (V == 1) {
        r[0] = p[0];
    } else {
#pragma unroll
        for (int k = 0; k < V; k += 2) {
            const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(p + k);
            r[k] = t.x;
            r[k + 1] = t.y;
        }
    }
}
// streaming load (evict-first in L1 and L2): for data read once, so that it does not push
// reused data out of L2
template <int V>
__device__ __forceinline__ void ldv_cs(const u64* p, u64 (&r)[V]) {
    if constexpr (V == 1) {
        r[0] = __ldcs(p);
    } else {
#pragma unroll
        for (int k = 0; k < V; k += 2) {
            const ulonglong2 t = __ldcs(reinterpret_cast<const ulonglong2*>(p + k));
            r[k] = t.x;
            r[k + 1] = t.y;
        }
    }
}
template <int V>
__device__ __forceinline__ void stv(u64* p, const u64 (&r)[V]) {
    if constexpr (V == 1) {
        p[0] = r[0];
    } else {
#pragma unroll
        for (int k = 0; k < V; k += 2) *reinterpret_cast<ulonglong2*>(p + k) = make_ulonglong2(r[k], r[k + 1]);
    }
}
#define EWV_BEGIN(n)                                                \
    const int j = V * (blockIdx.x * blockDim.x + threadIdx.x);      \
    if (j >= (n)) return;

template <int V>
__global__ void k_add(const u64* a, const u64* b, u64* o, const DevPrime* P, const int* ids, int lpp, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const u64 q = P[ids[limb % lpp]].m.q;
    const size_t off = (size_t)limb << logn;
    EWV_BEGIN(1 << logn)
    u64 x[V], y[V];
    ldv<V>(a + off + j, x);
    ldv<V>(b + off + j, y);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = add_mod(x[v], y[v], q);
    stv<V>(o + off + j, x);
}
template <int V>
__global__ void k_sub(const u64* a, const u64* b, u64* o, const DevPrime* P, const int* ids, int lpp, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const u64 q = P[ids[limb % lpp]].m.q;
    const size_t off = (size_t)limb << logn;
    EWV_BEGIN(1 << logn)
    u64 x[V], y[V];
    ldv<V>(a + off + j, x);
    ldv<V>(b + off + j, y);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = sub_mod(x[v], y[v], q);
    stv<V>(o + off + j, x);
}
template <int V>
__global__ void k_neg(const u64* a, u64* o, const DevPrime* P, const int* ids, int lpp, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const u64 q = P[ids[limb % lpp]].m.q;
    const size_t off = (size_t)limb << logn;
    EWV_BEGIN(1 << logn)
    u64 x[V];
    ldv<V>(a + off + j, x);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = neg_mod(x[v], q);
    stv<V>(o + off + j, x);
}
// bmod > 0: b is broadcast, row limb % bmod of b multiplies row limb of a (one plaintext times
// every polynomial of a batch of ciphertexts)
template <int V>
__global__ void k_mul(const u64* a, const u64* b, u64* o, const DevPrime* P, const int* ids, int lpp, int logn,
                      int bmod) {
    griddep_entry();
    const int limb = blockIdx.y;
    const DevMod m = P[ids[limb % lpp]].m;
    const size_t off = (size_t)limb << logn;
    const size_t boff = (size_t)(bmod ? limb % bmod : limb) << logn;
    EWV_BEGIN(1 << logn)
    u64 x[V], y[V];
    ldv<V>(a + off + j, x);
    ldv<V>(b + boff + j, y);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = mul_mod(x[v], y[v], m);
    stv<V>(o + off + j, x);
}
// tensor product of two ciphertexts: d0 = a0 b0, d1 = a0 b1 + a1 b0 (d [2][nl][N]), d2 = a1 b1
// (e [nl][N]); a, b [2][nl][N]; one pass over the nl limbs
// blockIdx.z: ciphertext t of a batch, its operands at a + t abs, b + t abs, d + t dbs, e + t ebs
template <int V>
__global__ void k_tensor(const u64* a, const u64* b, u64* d, u64* e, const DevPrime* P, const int* ids, int nl,
                         int logn, size_t abs, size_t dbs, size_t ebs) {
    griddep_entry();
    const int limb = blockIdx.y;
    const DevMod m = P[ids[limb]].m;
    const size_t off = (size_t)limb << logn, ps = (size_t)nl << logn;
    a += blockIdx.z * abs;
    b += blockIdx.z * abs;
    d += blockIdx.z * dbs;
    e += blockIdx.z * ebs;
    EWV_BEGIN(1 << logn)
    u64 a0[V], a1[V], b0[V], b1[V], d0[V], d1[V], d2[V];
    ldv<V>(a + off + j, a0);
    ldv<V>(a + ps + off + j, a1);
    ldv<V>(b + off + j, b0);
    ldv<V>(b + ps + off + j, b1);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        d0[v] = mul_mod(a0[v], b0[v], m);
        d1[v] = add_mod(mul_mod(a0[v], b1[v], m), mul_mod(a1[v], b0[v], m), m.q);
        d2[v] = mul_mod(a1[v], b1[v], m);
    }
    stv<V>(d + off + j, d0);
    stv<V>(d + ps + off + j, d1);
    stv<V>(e + off + j, d2);
}
template <int V>
__global__ void k_mul_acc(const u64* a, const u64* b, u64* o, const DevPrime* P, const int* ids, int lpp, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const DevMod m = P[ids[limb % lpp]].m;
    const size_t off = (size_t)limb << logn;
    EWV_BEGIN(1 << logn)
    u64 x[V], y[V], z[V];
    ldv<V>(a + off + j, x);
    ldv<V>(b + off + j, y);
    ldv<V>(o + off + j, z);
#pragma unroll
    for (int v = 0; v < V; ++v) z[v] = add_mod(z[v], mul_mod(x[v], y[v], m), m.q);
    stv<V>(o + off + j, z);
}
template <int V>
__global__ void k_mul_scalar(const u64* a, const u64* s, const u64* sp, u64* o, const DevPrime* P, const int* ids,
                             int lpp, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const u64 q = P[ids[r]].m.q;
    const u64 w = s[r], wp = sp[r];
    const size_t off = (size_t)limb << logn;
    EWV_BEGIN(1 << logn)
    u64 x[V];
    ldv<V>(a + off + j, x);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = mul_shoup(x[v], w, wp, q);
    stv<V>(o + off + j, x);
}
// per-limb scalars passed by value (no host-to-device copy, so the launch can be captured)
template <int V>
__global__ void k_mul_scalar_v(const u64* a, ScalarVec sv, u64* o, const DevPrime* P, const int* ids, int lpp,
                               size_t a_pstride, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const u64 q = P[ids[r]].m.q;
    const u64 w = sv.v[r], wp = sv.vp[r];
    const size_t off = (size_t)limb << logn;
    const size_t offa = a_pstride ? (size_t)(limb / lpp) * a_pstride + ((size_t)r << logn) : off;
    EWV_BEGIN(1 << logn)
    u64 x[V];
    ldv<V>(a + offa + j, x);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = mul_shoup(x[v], w, wp, q);
    stv<V>(o + off + j, x);
}
template <int V>
__global__ void k_lincomb(const __grid_constant__ kern::LinComb T, u64* __restrict__ o,
                          const DevPrime* __restrict__ P, const int* __restrict__ ids, int lpp, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const u64 q = P[ids[r]].m.q;
    const size_t off = (size_t)limb << logn;
    EWV_BEGIN(1 << logn)
    u64 acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0;
    for (int t = 0; t < T.n; ++t) {
        const u64 w = T.w[t][r], wp = T.wp[t][r];
        u64 x[V];
        ldv<V>(T.a[t] + off + j, x);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = add_mod(acc[v], mul_shoup(x[v], w, wp, q), q);
    }
    stv<V>(o + off + j, acc);
}
// ps > 0: row limb of a at (limb / lpp) ps + (limb % lpp) N (e.g. c0 of every ciphertext of a batch)
template <int V>
__global__ void k_add_scalar_v(u64* a, ScalarVec sv, const DevPrime* P, const int* ids, int lpp, int logn,
                               size_t ps) {
    griddep_entry();
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const u64 q = P[ids[r]].m.q;
    const u64 c = sv.v[r];
    const size_t off = ps ? (size_t)(limb / lpp) * ps + ((size_t)r << logn) : (size_t)limb << logn;
    EWV_BEGIN(1 << logn)
    u64 x[V];
    ldv<V>(a + off + j, x);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = add_mod(x[v], c, q);
    stv<V>(a + off + j, x);
}
template <int V>
__global__ void k_add_scalar(u64* a, const u64* vals, const DevPrime* P, const int* ids, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const u64 q = P[ids[limb]].m.q;
    const u64 c = vals[limb];
    const size_t off = (size_t)limb << logn;
    EWV_BEGIN(1 << logn)
    u64 x[V];
    ldv<V>(a + off + j, x);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = add_mod(x[v], c, q);
    stv<V>(a + off + j, x);
}
__global__ void k_small_to_rns(const int64_t* v, u64* o, const DevPrime* P, const int* ids, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const DevMod m = P[ids[limb]].m;
    const size_t off = (size_t)limb << logn;
    EW_LOOP(1 << logn) {
        const int64_t x = v[j];
        if (x >= 0) {
            o[off + j] = reduce64((u64)x, m);
        } else {
            const u64 r = reduce64((u64)(-(x + 1)) + 1ull, m);
            o[off + j] = r ? m.q - r : 0;
        }
    }
}
__global__ void k_automorph(const u64* a, u64* o, u64 g, int logn) {
    griddep_entry();
    const size_t off = (size_t)blockIdx.y << logn;
    EW_LOOP(1 << logn) o[off + j] = a[off + galois_src(j, g, logn)];
}
// o[limb][j] += s[limb % lpp] * a[limb][src_g(j)] (s null: plain add), NTT domain
template <int V>
__global__ void k_automorph_acc(const u64* a, u64* o, u64 g, const u64* s, const u64* sp, const DevPrime* P,
                                const int* ids, int lpp, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const u64 q = P[ids[r]].m.q;
    const size_t off = (size_t)limb << logn;
    EWV_BEGIN(1 << logn)
    u64 z[V];
    ldv<V>(o + off + j, z);
    if (s) {
        const u64 w = s[r], wp = sp[r];
#pragma unroll
        for (int v = 0; v < V; ++v) z[v] = add_mod(z[v], mul_shoup(a[off + galois_src(j + v, g, logn)], w, wp, q), q);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) z[v] = add_mod(z[v], a[off + galois_src(j + v, g, logn)], q);
    }
    stv<V>(o + off + j, z);
}
__global__ void k_imult(const u64* a, u64* o, const DevPrime* P, const int* ids, int lpp, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const DevPrime* pr = P + ids[limb % lpp];
    const u64 q = pr->m.q;
    // X^{N/2} at psi^(2r+1): psi^{N/2} when r is even, -psi^{N/2} when r is odd;
    // psi^{N/2} = tw[1] since rev(1) = N/2
    const u64 w = pr->tw[1].x, wp = pr->tw[1].y;
    const size_t off = (size_t)limb << logn;
    EW_LOOP(1 << logn) {
        u64 v = mul_shoup(a[off + j], w, wp, q);
        unsigned r = brev_bits(j, logn);
        o[off + j] = (r & 1) ? neg_mod(v, q) : v;
    }
}
template <int V>
__global__ void k_lift_centred(const u64* src, u64 qs, u64* o, const DevPrime* P, const int* ids, int lpp,
                               size_t src_pstride, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const DevMod t = P[ids[limb % lpp]].m;
    const size_t off = (size_t)limb << logn;
    const u64* sr = src + (size_t)(limb / lpp) * src_pstride;
    EWV_BEGIN(1 << logn)
    u64 x[V];
    ldv<V>(sr + j, x);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = centred_to(x[v], qs, t);
    stv<V>(o + off + j, x);
}
template <int V>
__global__ void k_sub_mul2_scalar(const u64* a, const u64* b, ScalarVec s1, const u64* s2, const u64* s2p, u64* o,
                                  const DevPrime* P, const int* ids, int lpp, size_t a_pstride, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const u64 q = P[ids[r]].m.q;
    const u64 w1 = s1.v[r], w1p = s1.vp[r], w2 = s2[r], w2p = s2p[r];
    const size_t off = (size_t)limb << logn;
    const size_t offa = a_pstride ? (size_t)(limb / lpp) * a_pstride + ((size_t)r << logn) : off;
    EWV_BEGIN(1 << logn)
    u64 x[V], y[V];
    ldv<V>(a + offa + j, x);
    ldv<V>(b + off + j, y);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = sub_mod(mul_shoup(x[v], w1, w1p, q), mul_shoup(y[v], w2, w2p, q), q);
    stv<V>(o + off + j, x);
}
template <int V>
__global__ void k_sub_mul_scalar(const u64* a, const u64* b, const u64* s, const u64* sp, u64* o,
                                 const DevPrime* P, const int* ids, int lpp, size_t a_pstride, int logn) {
    griddep_entry();
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const u64 q = P[ids[r]].m.q;
    const u64 w = s[r], wp = sp[r];
    const size_t off = (size_t)limb << logn;
    const size_t offa = a_pstride ? (size_t)(limb / lpp) * a_pstride + ((size_t)r << logn) : off;
    EWV_BEGIN(1 << logn)
    u64 x[V], y[V];
    ldv<V>(a + offa + j, x);
    ldv<V>(b + off + j, y);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = mul_shoup(sub_mod(x[v], y[v], q), w, wp, q);
    stv<V>(o + off + j, x);
}

// ------------------------------------------------- BSGS inner products ----
// o[g][poly][limb] = sum_b a_b[poly][limb] * p_{g,b}[limb] for NG giant steps at once: each
// baby value is loaded once and multiplied into every giant step's sum; the products are
// summed exactly in 128 bits (each < 2^122, at most 32 terms) and reduced once.
// blockIdx.y = row * nbt + t: ciphertext t of a batch (babies at T.a[b] + t astr, outputs at
// T.o[g] + t ostr; the diagonals are shared and read by neighbouring CTAs)
template <int V, int NG>
__global__ void k_bsgs_inner_giants(kern::BsgsGiants T, const DevPrime* __restrict__ primes, int nl,
                                    const int* __restrict__ ids, int logn, int nbt, size_t astr, size_t ostr) {
    griddep_entry();
    const int t = blockIdx.y % nbt;
    const int limb = blockIdx.y / nbt;     // 0 .. 2 nl - 1, polynomial-major
    const int r = limb % nl;
    const DevPrime P = primes[ids[r]];
    const size_t offa = t * astr + ((size_t)limb << logn), offo = t * ostr + ((size_t)limb << logn);
    const size_t offp = (size_t)r << logn;
    EWV_BEGIN(1 << logn)
    u64 lo[NG][V], hi[NG][V];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int v = 0; v < V; ++v) lo[g][v] = hi[g][v] = 0;
    for (int b = 0; b < T.nb; ++b) {
        u64 x[V];
        ldv<V>(T.a[b] + offa + j, x);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const u64* pg = T.p[g][b];
            if (!pg) continue;
            u64 y[V];
            ldv<V>(pg + offp + j, y);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const u64 pl = x[v] * y[v], ph = __umul64hi(x[v], y[v]);
                lo[g][v] += pl;
                hi[g][v] += ph + (lo[g][v] < pl ? 1ull : 0ull);
            }
        }
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        u64 res[V];
#pragma unroll
        for (int v = 0; v < V; ++v) res[v] = reduce128_lazy(hi[g][v], lo[g][v], P);
        if ((T.acc >> g) & 1u) {
            u64 prev[V];
            ldv<V>(T.o[g] + offo + j, prev);
#pragma unroll
            for (int v = 0; v < V; ++v) res[v] = add_mod(res[v], prev[v], P.m.q);
        }
        stv<V>(T.o[g] + offo + j, res);
    }
}

// Baby rotations fused with the giant-step inner sums (see kern::bsgs_fused): per baby the
// key-switch product is summed in 128 bits and reduced, the automorphed c0 term added, and the
// reduced baby multiplied into every giant step's 128-bit sum; the babies stay in registers.
// Same arithmetic as k_ks_inner_d followed by k_bsgs_inner_giants, so the same residues.
// The next baby's operands (key words, gathered digit words, c0, diagonal words) are copied
// into shared memory by per-thread asynchronous copies while the current baby is computed:
// two stages of NS words per thread, so the memory latency of a baby overlaps the arithmetic
// of the previous one without holding the words in registers (a version loading them into
// registers ran 1.7x slower on a top-level CtoS level, latency bound at 36% warp occupancy).
__device__ __forceinline__ void cp_async8(u64* dst_smem, const u64* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int NDIG, int NG>
__global__ void __launch_bounds__(256, 3)
    k_bsgs_fused_async(const __grid_constant__ kern::BsgsFused T, const u64* __restrict__ D,
                       const u64* __restrict__ c0, const u64* __restrict__ c1, int nl, int next,
                       const int* __restrict__ ext_ids, const u64* __restrict__ s0, const u64* __restrict__ s0p,
                       const DevPrime* __restrict__ P, int logn, size_t kstride, kern::KsBatch bt) {
    griddep_entry();
    constexpr int NS = 3 * NDIG + 2 + NG;       // kb, ka, D per digit; c0 (gathered or row); c1 row; diagonals
    extern __shared__ u64 sbuf[];               // [2][NS][256]
    const int e = blockIdx.y;
    const int id = ext_ids[e];
    const DevPrime pr = P[id];
    const u64 q = pr.m.q;
    const size_t n = (size_t)1 << logn;
    const bool qrow = e < nl;
    const u64 w = qrow ? s0[e] : 0, wp = qrow ? s0p[e] : 0;
    const int tid = threadIdx.x;
    // ciphertext t of a batch (fastest varying, so that the CTAs reading the same key and diagonal
    // words run side by side and share them through L2): D + t dstr, c0 / c1 + t xstr, outputs
    // + t ostr
    const int t = blockIdx.x % bt.nb;
    const int j = (blockIdx.x / bt.nb) * 256 + tid;
    if (j >= (int)n) return;
    D += t * bt.dstr;
    c0 += t * bt.xstr;
    c1 += t * bt.xstr;
    auto slot = [&](int st, int k) -> u64* { return sbuf + ((size_t)(st * NS + k) << 8) + tid; };
    auto issue = [&](int b, int st) {
        if (!T.kb[b]) {
            if (qrow) {
                cp_async8(slot(st, 3 * NDIG), c0 + (size_t)e * n + j);
                cp_async8(slot(st, 3 * NDIG + 1), c1 + (size_t)e * n + j);
            }
        } else {
            const unsigned src = galois_src(j, T.gal[b], logn);
#pragma unroll
            for (int d = 0; d < NDIG; ++d) {
                const size_t kk = d * kstride + (size_t)id * n + j;
                cp_async8(slot(st, d), T.kb[b] + kk);
                cp_async8(slot(st, NDIG + d), T.ka[b] + kk);
                cp_async8(slot(st, 2 * NDIG + d), D + ((size_t)d * next + e) * n + src);
            }
            if (qrow) cp_async8(slot(st, 3 * NDIG), c0 + (size_t)e * n + src);
        }
#pragma unroll
        for (int g = 0; g < NG; ++g)
            if (T.p[g][b]) cp_async8(slot(st, 3 * NDIG + 2 + g), T.p[g][b] + (size_t)e * n + j);
        cp_async_commit();
    };
    u64 lob[NG], hib[NG], loa[NG], hia[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) lob[g] = hib[g] = loa[g] = hia[g] = 0;
    issue(0, 0);
    if (T.nb > 1) issue(1, 1);
    else cp_async_commit();
    for (int b = 0; b < T.nb; ++b) {
        const int st = b & 1;
        cp_async_wait<1>();                          // the group of baby b has landed
        u64 rb, ra;
        if (!T.kb[b]) {
            rb = qrow ? mul_shoup(*slot(st, 3 * NDIG), w, wp, q) : 0;
            ra = qrow ? mul_shoup(*slot(st, 3 * NDIG + 1), w, wp, q) : 0;
        } else {
            u64 bl = 0, bh = 0, al = 0, ah = 0;
#pragma unroll
            for (int d = 0; d < NDIG; ++d) {
                const u64 x = *slot(st, 2 * NDIG + d), yb = *slot(st, d), ya = *slot(st, NDIG + d);
                mac128(bl, bh, x, yb);
                mac128(al, ah, x, ya);
            }
            rb = reduce128_lazy(bh, bl, pr);
            ra = reduce128_lazy(ah, al, pr);
            if (qrow) rb = add_mod(rb, mul_shoup(*slot(st, 3 * NDIG), w, wp, q), q);
        }
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            if (!T.p[g][b]) continue;
            const u64 y = *slot(st, 3 * NDIG + 2 + g);
            mac128(lob[g], hib[g], rb, y);
            mac128(loa[g], hia[g], ra, y);
        }
        if (b + 2 < T.nb) issue(b + 2, st);          // this stage has been read
        else cp_async_commit();                      // keep one group per iteration
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        u64 vb = reduce128_lazy(hib[g], lob[g], pr), va = reduce128_lazy(hia[g], loa[g], pr);
        u64* ob = T.o[g] + t * bt.ostr + (size_t)e * n + j;
        u64* oa = T.o[g] + t * bt.ostr + ((size_t)next + e) * n + j;
        if ((T.acc >> g) & 1u) {
            vb = add_mod(vb, *ob, q);
            va = add_mod(va, *oa, q);
        }
        *ob = vb;
        *oa = va;
    }
}

// ------------------------------------------------------- base conversion ----
// y_m = sum_i [x_i * qhat_i^{-1}]_{q_i} * (qhat_i mod p_m)  (no correction term), or, for an
// exact table, minus v (Q mod p_m) with v = round(sum_i xhat_i / q_i) (Halevi, Polyakov,
// Shoup 2019), evaluated in 58-bit fixed point (conv_round_term): y then represents the
// centred remainder of x mod Q, up to a rounding error that matters only within 2^-53 of a
// half-integer.
// One thread per coefficient; grid.z walks over (job, group of MC <= CONV_OUT outputs), so
// the digits of one ModUp (or the two halves of one ModDown) share a launch.  The products
// are summed exactly in 128 bits (each < 2^122, at most 16 terms) and reduced once:
// (H 2^64 + L) mod p = H (2^64 mod p) + L mod p.  The output loop is unrolled so that the
// MC independent accumulations interleave.
constexpr int MAX_CONV_IN = 16;
constexpr int CONV_OUT = 8;
// MAXIN: compile-time bound on the jobs' input counts (4, 8 or 16), so that the unrolled
// input loops carry no predicated-off iterations for the common 7- and 8-limb conversions.
// SPLIT (every modulus below 2^60, MAXIN <= 8): x = xu 2^30 + xl, c = cu 2^30 + cl; the four
// partial products (each < 2^60) go into three 64-bit sums by one 32x32->64 multiply-add
// each (at most 16 terms per sum: no overflow); the 128-bit total ll + m 2^30 + hh 2^60 is
// then reduced as in the general path.
// MC: outputs per CTA group (4..8), chosen per launch to leave the fewest idle output slots.
template <int MAXIN, bool SPLIT, int MC>
__global__ void __launch_bounds__(256, (MC <= 6 ? 4 : 3)) k_base_convert(kern::ConvJobs J, const DevPrime* __restrict__ P, int logn) {
    griddep_entry();
    __shared__ u64 s_qi[MAX_CONV_IN], s_qinv[MAX_CONV_IN], s_qinvp[MAX_CONV_IN];
    __shared__ u64 s_c[CONV_OUT][MAX_CONV_IN];
    __shared__ DevPrime s_pm[CONV_OUT];
    __shared__ int s_row[CONV_OUT];
    __shared__ u64 s_invm[MAX_CONV_IN];
    __shared__ int s_invs[MAX_CONV_IN];
    __shared__ u64 s_corr[CONV_OUT];
    __shared__ uint2 s_c2[CONV_OUT][MAXIN];     // SPLIT: (c mod 2^30, c >> 30)
    // which job and output group this CTA serves
    int z = blockIdx.z, jb = 0;
    while (jb < J.n - 1 && z >= J.job[jb].ngroups) {
        z -= J.job[jb].ngroups;
        ++jb;
    }
    const kern::ConvJob& job = J.job[jb];
    const int nin = job.nin, nout = job.nout;
    const int m0 = z * MC;
    const int mcount = min(MC, nout - m0);
    const int tid = threadIdx.x;
    const bool exact = job.inv_q != nullptr;
    if (tid < nin) {
        s_qi[tid] = P[job.in_ids[tid]].m.q;
        s_qinv[tid] = job.qinv[tid];
        s_qinvp[tid] = job.qinv[nin + tid];
        s_invm[tid] = exact ? job.inv_q[tid] : 0;
        s_invs[tid] = exact ? (int)job.inv_q[nin + tid] : 64;
    }
    if (tid < CONV_OUT * MAX_CONV_IN) {
        const int m = tid / MAX_CONV_IN, i = tid % MAX_CONV_IN;
        const u64 c = (m < mcount && i < nin) ? job.qmod[(size_t)(m0 + m) * nin + i] : 0;
        s_c[m][i] = c;
        if (SPLIT && i < MAXIN) s_c2[m][i] = make_uint2((unsigned)(c & ((1ull << 30) - 1)), (unsigned)(c >> 30));
    }
    if (tid < mcount) {
        s_pm[tid] = P[job.out_ids[m0 + tid]];
        s_row[tid] = job.out_rows[m0 + tid];
        s_corr[tid] = exact ? job.corr[m0 + tid] : 0;
    }
    __syncthreads();
    const u64* in = job.in + blockIdx.y * job.in_pstride;
    u64* out = job.out + blockIdx.y * job.out_pstride;
    const int j = blockIdx.x * blockDim.x + tid;
    if (j >= (1 << logn)) return;
    const size_t n = (size_t)1 << logn;
    u64 xh[MAXIN];
#pragma unroll
    for (int i = 0; i < MAXIN; ++i)
        if (i < nin) xh[i] = job.prescaled ? in[i * n + j] : mul_shoup(in[i * n + j], s_qinv[i], s_qinvp[i], s_qi[i]);
    u64 lo[MC], hi[MC];
    if (SPLIT) {
        constexpr u64 M30 = (1ull << 30) - 1;
        u64 ll[MC], mm[MC], hh[MC];
#pragma unroll
        for (int m = 0; m < MC; ++m) ll[m] = mm[m] = hh[m] = 0;
#pragma unroll
        for (int i = 0; i < MAXIN; ++i) {
            if (i < nin) {
                const unsigned xl = (unsigned)(xh[i] & M30), xu = (unsigned)(xh[i] >> 30);
#pragma unroll
                for (int m = 0; m < MC; ++m) {
                    const uint2 cc = s_c2[m][i];
                    ll[m] += (u64)xl * cc.x;
                    mm[m] += (u64)xl * cc.y;
                    mm[m] += (u64)xu * cc.x;
                    hh[m] += (u64)xu * cc.y;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < MC; ++m) {
            u64 l = ll[m], h = (mm[m] >> 34) + (hh[m] >> 4);
            const u64 t1 = mm[m] << 30;
            l += t1;
            h += l < t1 ? 1ull : 0ull;
            const u64 t2 = hh[m] << 60;
            l += t2;
            h += l < t2 ? 1ull : 0ull;
            lo[m] = l;
            hi[m] = h;
        }
    } else {
#pragma unroll
        for (int m = 0; m < MC; ++m) lo[m] = hi[m] = 0;
#pragma unroll
        for (int i = 0; i < MAXIN; ++i) {
            if (i < nin) {
#pragma unroll
                for (int m = 0; m < MC; ++m) {
                    const u64 c = s_c[m][i];
                    const u64 pl = xh[i] * c, ph = __umul64hi(xh[i], c);
                    lo[m] += pl;
                    hi[m] += ph + (lo[m] < pl ? 1ull : 0ull);
                }
            }
        }
    }
    if (exact) {
        u64 f = 0;
#pragma unroll
        for (int i = 0; i < MAXIN; ++i)
            if (i < nin) f += conv_round_term(xh[i], s_invm[i], s_invs[i]);
        const u64 v = conv_round_finish(f);
#pragma unroll
        for (int m = 0; m < MC; ++m) {
            const u64 pl = v * s_corr[m], ph = __umul64hi(v, s_corr[m]);
            lo[m] += pl;
            hi[m] += ph + (lo[m] < pl ? 1ull : 0ull);
        }
    }
#pragma unroll
    for (int m = 0; m < MC; ++m)
        if (m < mcount) out[(size_t)s_row[m] * n + j] = reduce128_lazy(hi[m], lo[m], s_pm[m]);
}

// ---------------------------------------------------- key-switch product ----
template <bool ACC, int V>
__global__ void k_ks_inner(const u64* __restrict__ D, int ndig, int next, const int* __restrict__ ext_ids,
                           const u64* __restrict__ kb, const u64* __restrict__ ka, u64* __restrict__ ob,
                           u64* __restrict__ oa, const DevPrime* __restrict__ P, int logn, u64 g, size_t kstride) {
    griddep_entry();
    const int e = blockIdx.y;
    const int id = ext_ids[e];
    const DevMod m = P[id].m;
    const size_t n = (size_t)1 << logn;
    EWV_BEGIN(1 << logn)
    unsigned src[V];
#pragma unroll
    for (int v = 0; v < V; ++v) src[v] = g == 1 ? (unsigned)(j + v) : galois_src(j + v, g, logn);
    u64 accb[V], acca[V];
#pragma unroll
    for (int v = 0; v < V; ++v) accb[v] = acca[v] = 0;
    for (int d = 0; d < ndig; ++d) {
        const u64* Dd = D + ((size_t)d * next + e) * n;
        const size_t kk = d * kstride + (size_t)id * n + j;
        u64 yb[V], ya[V];
        ldv<V>(kb + kk, yb);
        ldv<V>(ka + kk, ya);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const u64 x = Dd[src[v]];
            accb[v] = add_mod(accb[v], mul_mod(x, yb[v], m), m.q);
            acca[v] = add_mod(acca[v], mul_mod(x, ya[v], m), m.q);
        }
    }
    if (ACC) {
        u64 pb[V], pa[V];
        ldv<V>(ob + (size_t)e * n + j, pb);
        ldv<V>(oa + (size_t)e * n + j, pa);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            accb[v] = add_mod(accb[v], pb[v], m.q);
            acca[v] = add_mod(acca[v], pa[v], m.q);
        }
    }
    stv<V>(ob + (size_t)e * n + j, accb);
    stv<V>(oa + (size_t)e * n + j, acca);
}

// The same product for a digit count fixed at compile time: every digit's key words and
// gathered input are loaded before any arithmetic, the products are summed exactly in 128 bits
// (each < 2^122, at most 4 terms) and reduced once per output word.
// A batch of bt.nb key switches with the same key: ciphertext t's digits at D + t dstr, its
// outputs at ob / oa + t ostr, its x0 / x1 at + t xstr.  The ciphertext index is the fastest
// varying part of blockIdx.x, so the CTAs that read the same key words run side by side and
// all but the first find them in L2: the key streams from HBM about once per batch.
template <bool ACC, int V, int NDIG>
__global__ void k_ks_inner_d(const u64* __restrict__ D, int next, const int* __restrict__ ext_ids,
                             const u64* __restrict__ kb, const u64* __restrict__ ka, u64* __restrict__ ob,
                             u64* __restrict__ oa, const DevPrime* __restrict__ P, int logn, u64 g, size_t kstride,
                             const u64* __restrict__ x0, const u64* __restrict__ x1, int x0rows,
                             const u64* __restrict__ s0, const u64* __restrict__ s0p, kern::KsBatch bt) {
    griddep_entry();
    const int e = blockIdx.y;
    const int id = ext_ids[e];
    const DevPrime pr = P[id];
    const size_t n = (size_t)1 << logn;
    const int t = blockIdx.x % bt.nb;
    const int j = V * ((blockIdx.x / bt.nb) * blockDim.x + threadIdx.x);
    if (j >= (int)n) return;
    D += t * bt.dstr;
    ob += t * bt.ostr;
    oa += t * bt.ostr;
    if (x0) x0 += t * bt.xstr;
    if (x1) x1 += t * bt.xstr;
    unsigned src[V];
#pragma unroll
    for (int v = 0; v < V; ++v) src[v] = g == 1 ? (unsigned)(j + v) : galois_src(j + v, g, logn);
    u64 x[NDIG][V], yb[NDIG][V], ya[NDIG][V];
#pragma unroll
    for (int d = 0; d < NDIG; ++d) {
        const u64* Dd = D + ((size_t)d * next + e) * n;
        const size_t kk = d * kstride + (size_t)id * n + j;
        if (bt.nb == 1) {
            ldv_cs<V>(kb + kk, yb[d]);   // each key word is read once per key switch: keep the
            ldv_cs<V>(ka + kk, ya[d]);   // raised digits, which every rotation re-reads, in L2
        } else {
            ldv<V>(kb + kk, yb[d]);      // the other ciphertexts of the batch read them next
            ldv<V>(ka + kk, ya[d]);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) x[d][v] = Dd[src[v]];
    }
    u64 rb[V], ra[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        u64 bl = 0, bh = 0, al = 0, ah = 0;
#pragma unroll
        for (int d = 0; d < NDIG; ++d) {
            const u64 pbl = x[d][v] * yb[d][v], pal = x[d][v] * ya[d][v];
            bh += __umul64hi(x[d][v], yb[d][v]);
            ah += __umul64hi(x[d][v], ya[d][v]);
            bl += pbl;
            bh += bl < pbl ? 1ull : 0ull;
            al += pal;
            ah += al < pal ? 1ull : 0ull;
        }
        rb[v] = reduce128_lazy(bh, bl, pr);
        ra[v] = reduce128_lazy(ah, al, pr);
    }
    if (ACC) {
        u64 pb[V], pa[V];
        ldv<V>(ob + (size_t)e * n + j, pb);
        ldv<V>(oa + (size_t)e * n + j, pa);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            rb[v] = add_mod(rb[v], pb[v], pr.m.q);
            ra[v] = add_mod(ra[v], pa[v], pr.m.q);
        }
    }
    if (x0 && e < x0rows) {
        const u64* xr = x0 + (size_t)e * n;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            u64 t = xr[src[v]];
            if (s0) t = mul_shoup(t, s0[e], s0p[e], pr.m.q);
            rb[v] = add_mod(rb[v], t, pr.m.q);
        }
        if (x1) {
            const u64* yr = x1 + (size_t)e * n;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                u64 t = yr[src[v]];
                if (s0) t = mul_shoup(t, s0[e], s0p[e], pr.m.q);
                ra[v] = add_mod(ra[v], t, pr.m.q);
            }
        }
    }
    stv<V>(ob + (size_t)e * n + j, rb);
    stv<V>(oa + (size_t)e * n + j, ra);
}

// o += a * s[limb % lpp] (Shoup pairs s, sp)
template <int V>
// o_ps > 0: row limb of o at (limb / lpp) o_ps + (limb % lpp) N (a contiguous)
__global__ void k_mul_scalar_acc(const u64* a, const u64* s, const u64* sp, u64* o, const DevPrime* P, const int* ids,
                                 int lpp, int logn, size_t o_ps) {
    griddep_entry();
    const int limb = blockIdx.y;
    const int r = limb % lpp;
    const u64 q = P[ids[r]].m.q;
    const u64 w = s[r], wp = sp[r];
    const size_t off = (size_t)limb << logn;
    const size_t ooff = o_ps ? (size_t)(limb / lpp) * o_ps + ((size_t)r << logn) : off;
    EWV_BEGIN(1 << logn)
    u64 x[V], z[V];
    ldv<V>(a + off + j, x);
    ldv<V>(o + ooff + j, z);
#pragma unroll
    for (int v = 0; v < V; ++v) z[v] = add_mod(z[v], mul_shoup(x[v], w, wp, q), q);
    stv<V>(o + ooff + j, z);
}

// ------------------------------------------------------------ sampling ----
__device__ __forceinline__ u64 d_mix(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ u64 d_word(u64 key, u64 i) { return d_mix(key + (i + 1) * 0x9E3779B97F4A7C15ULL); }

__global__ void k_sample_uniform(u64* o, const DevPrime* P, const int* ids, int logn, u64 key) {
    griddep_entry();
    const int limb = blockIdx.y;
    const int id = ids[limb];
    const DevMod m = P[id].m;
    const u64 two64 = barrett_reduce128(1, 0, m);   // 2^64 mod q
    const size_t off = (size_t)limb << logn;
    EW_LOOP(1 << logn) {
        const u64 k = ((u64)id << logn) + (u64)j;
        const u64 w1 = d_word(key, 2 * k), w2 = d_word(key, 2 * k + 1);
        o[off + j] = add_mod(mul_mod(reduce64(w1, m), two64, m), reduce64(w2, m), m.q);
    }
}
__global__ void k_sample_small(int64_t* o, int logn, u64 key, int kind, const u64* gauss) {
    griddep_entry();
    EW_LOOP(1 << logn) {
        const u64 w = d_word(key, (u64)j);
        if (kind == 0) {
            o[j] = (int64_t)(w % 3ull) - 1;
        } else {
            const u64 u = w >> 1;
            int k = 0;
            while (k < 38 && u >= gauss[k]) ++k;
            o[j] = (int64_t)k - 19;
        }
    }
}

}  // namespace

// ------------------------------------------------------------- launchers ---
namespace kern {

#define LAUNCH_CHECK() CUDA_CHECK(cudaGetLastError())

void ntt_forward(const ckks_ctx* c, u64* data, int nlimbs, const int* ids, int lpp, size_t pstride) {
    if (nlimbs <= 0) return;
    if (pstride == 0) pstride = (size_t)lpp * c->n;
    if (c->logn == 16) {
        launch_ntt_transform<false>(c, data, nlimbs, ids, lpp, pstride);
        LAUNCH_CHECK();
        return;
    }
    for (const PassPlan& p : ntt_passes(c->logn)) launch_pass<false>(c, data, nlimbs, ids, lpp, pstride, p, 0);
    LAUNCH_CHECK();
}

// Time every NTT variant (forward + inverse) on scratch limbs of each size class and keep the
// fastest per class in ctx->ntt_choice.  Results are identical for every variant.
void autotune_ntt(ckks_ctx* c, int reps) {
    if (c->logn != 16) return;
    const int sizes[8] = {1, 2, 7, 14, 24, 48, 96, 192};
    DevBuf buf((size_t)192 << 16, c->stream);
    CUDA_CHECK(cudaMemsetAsync(buf.ptr, 0, ((size_t)192 << 16) * 8, c->stream));
    std::vector<int> ids(192);
    for (int i = 0; i < 192; ++i) ids[i] = i % c->nall;
    DevBuf dids(96, c->stream);
    CUDA_CHECK(cudaMemcpyAsync(dids.ptr, ids.data(), 192 * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int k = 0; k < 8; ++k) {
        const int nl = sizes[k];
        float best = 1e30f;
        int bestv = -1;
        for (int v = 0; v < NTT_NVARIANTS; ++v) {
            for (int w = 0; w < 2; ++w) {   // warm up, then time
                cudaEventRecord(e0, c->stream);
                for (int r = 0; r < reps; ++r) {
                    const int* d = (const int*)dids.ptr;
                    launch_ntt_variant<false>(c, v, buf.ptr, nl, d, nl, (size_t)nl << 16, nullptr);
                    launch_ntt_variant<true>(c, v, buf.ptr, nl, d, nl, (size_t)nl << 16, nullptr);
                }
                cudaEventRecord(e1, c->stream);
                CUDA_CHECK(cudaEventSynchronize(e1));
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bestv = v;
            }
        }
        c->ntt_choice[k] = bestv;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LAUNCH_CHECK();
}

void ntt_forward_list(const ckks_ctx* c, u64* data, int nlimbs, const int* off, const int* ids, int nb,
                      size_t bstride) {
    if (nlimbs <= 0 || nb <= 0) return;
    CK_CHECK(c->logn == 16, CKKS_EINVAL, "limb-list NTT needs N = 2^16");
    launch_ntt_transform<false>(c, data, nlimbs * nb, ids, nlimbs, bstride, off);
    LAUNCH_CHECK();
}

template <int V>
static void launch_bsgs_giants(const ckks_ctx* c, const BsgsGiants& t, int nl, const int* ids, const KsBatch& bt) {
    const dim3 grid = ewv_grid(c->n, 2 * nl * bt.nb, V);
#define GIANTS_CASE(NG)                                                                                         \
    klaunch(c, k_bsgs_inner_giants<V, NG>, grid, EW_THREADS, 0, t, c->d_primes, nl, ids, c->logn, bt.nb, bt.dstr, \
            bt.ostr)
    switch (t.ng) {
        case 1: GIANTS_CASE(1); break;
        case 2: GIANTS_CASE(2); break;
        case 3: GIANTS_CASE(3); break;
        case 4: GIANTS_CASE(4); break;
        case 5: GIANTS_CASE(5); break;
        case 6: GIANTS_CASE(6); break;
        case 7: GIANTS_CASE(7); break;
        default: GIANTS_CASE(8); break;
    }
#undef GIANTS_CASE
}

void bsgs_inner_giants(const ckks_ctx* c, const BsgsGiants& t, int nl, const int* ids, const KsBatch& bt) {
    CK_CHECK(t.nb >= 1 && t.nb <= BsgsGiants::MAXB && t.ng >= 1 && t.ng <= BsgsGiants::MAXG, CKKS_EINVAL,
             "1..32 baby steps and 1..8 giant steps per inner-sum launch");
    int terms = 0;
    bool vec = true;
    for (int b = 0; b < t.nb; ++b) vec = vec && al16(t.a[b]);
    for (int g = 0; g < t.ng; ++g) {
        vec = vec && al16(t.o[g]);
        for (int b = 0; b < t.nb; ++b)
            if (t.p[g][b]) {
                ++terms;
                vec = vec && al16(t.p[g][b]);
            }
    }
    {
        // algorithmic bytes: every baby (2 polynomials) once, every diagonal once, each giant's
        // output written (and read when accumulating)
        int accs = 0;
        for (int g = 0; g < t.ng; ++g) accs += (t.acc >> g) & 1u;
        KTimer kt_(c, "bsgs_inner", (bt.nb * (2.0 * t.nb + 2.0 * t.ng + 2.0 * accs) + terms) * nl * c->n * 8.0);
        if (vec)
            launch_bsgs_giants<2>(c, t, nl, ids, bt);
        else
            launch_bsgs_giants<1>(c, t, nl, ids, bt);
    }
    LAUNCH_CHECK();
}

template <int NDIG, int NG>
static void launch_bsgs_async_one(const ckks_ctx* c, const BsgsFused& t, const u64* D, const u64* c0,
                                  const u64* c1, int nl, int next, const int* ext, const u64* s, const u64* sp,
                                  const KsBatch& bt) {
    constexpr int NS = 3 * NDIG + 2 + NG;
    const size_t smem = 2 * (size_t)NS * 256 * sizeof(u64);
    static std::atomic<unsigned> done{0};
    allow_dynamic_smem((const void*)k_bsgs_fused_async<NDIG, NG>, (int)smem, done);
    const dim3 grid((c->n + 255) / 256 * bt.nb, next);
    klaunch(c, k_bsgs_fused_async<NDIG, NG>, grid, 256, smem, t, D, c0, c1, nl, next, ext, s, sp, c->d_primes,
            c->logn, (size_t)c->nall << c->logn, bt);
}

template <int NDIG>
static void launch_bsgs_async_g(const ckks_ctx* c, const BsgsFused& t, const u64* D, const u64* c0, const u64* c1,
                                int nl, int next, const int* ext, const u64* s, const u64* sp, const KsBatch& bt) {
    switch (t.ng) {
        case 1: launch_bsgs_async_one<NDIG, 1>(c, t, D, c0, c1, nl, next, ext, s, sp, bt); break;
        case 2: launch_bsgs_async_one<NDIG, 2>(c, t, D, c0, c1, nl, next, ext, s, sp, bt); break;
        case 3: launch_bsgs_async_one<NDIG, 3>(c, t, D, c0, c1, nl, next, ext, s, sp, bt); break;
        default: launch_bsgs_async_one<NDIG, 4>(c, t, D, c0, c1, nl, next, ext, s, sp, bt); break;
    }
}

static void launch_bsgs_async(const ckks_ctx* c, const BsgsFused& t, const u64* D, const u64* c0, const u64* c1,
                              int nl, int next, const int* ext, const u64* s, const u64* sp, const KsBatch& bt) {
    switch (t.ndig) {
        case 1: launch_bsgs_async_g<1>(c, t, D, c0, c1, nl, next, ext, s, sp, bt); break;
        case 2: launch_bsgs_async_g<2>(c, t, D, c0, c1, nl, next, ext, s, sp, bt); break;
        case 3: launch_bsgs_async_g<3>(c, t, D, c0, c1, nl, next, ext, s, sp, bt); break;
        default: launch_bsgs_async_g<4>(c, t, D, c0, c1, nl, next, ext, s, sp, bt); break;
    }
}

void bsgs_fused(const ckks_ctx* c, const BsgsFused& t, const u64* D, const u64* c0, const u64* c1, int nl,
                int next, const int* ext_ids, const u64* s, const u64* sp, const KsBatch& bt) {
    CK_CHECK(t.nb >= 1 && t.nb <= BsgsFused::MAXB && t.ng >= 1 && t.ng <= BsgsFused::MAXG && t.ndig >= 1 &&
                 t.ndig <= 4, CKKS_EINVAL, "fused BSGS: 1..32 babies, 1..4 giant steps, 1..4 digits");
    int terms = 0, rots = 0;
    for (int b = 0; b < t.nb; ++b) {
        if (t.kb[b]) ++rots;
        for (int g = 0; g < t.ng; ++g)
            if (t.p[g][b]) ++terms;
    }
    int accs = 0;
    for (int g = 0; g < t.ng; ++g) accs += (t.acc >> g) & 1u;
    {
        // algorithmic bytes: per rotation the digits, both key halves and c0 on the Q rows; the
        // identity's c0 and c1; every diagonal once; each giant's output (read when accumulating)
        // (a batch reads the keys and diagonals once, and its ciphertexts' own words each)
        const double shared = (double)rots * 2.0 * t.ndig + terms;
        const double own = (double)rots * (t.ndig * next + nl) / next + (t.nb - rots) * 2.0 * nl / next +
                           2.0 * t.ng + 2.0 * accs;
        KTimer kt_(c, "bsgs_fused", (shared + bt.nb * own) * next * c->n * 8.0);
        launch_bsgs_async(c, t, D, c0, c1, nl, next, ext_ids, s, sp, bt);
    }
    LAUNCH_CHECK();
}

void ntt_inverse(const ckks_ctx* c, u64* data, int nlimbs, const int* ids, int lpp, size_t pstride, const u64* osc) {
    if (nlimbs <= 0) return;
    if (pstride == 0) pstride = (size_t)lpp * c->n;
    if (c->logn == 16) {
        launch_ntt_transform<true>(c, data, nlimbs, ids, lpp, pstride, nullptr, osc);
        LAUNCH_CHECK();
        return;
    }
    std::vector<PassPlan> ps = ntt_passes(c->logn);
    for (int i = (int)ps.size() - 1; i >= 0; --i)
        launch_pass<true>(c, data, nlimbs, ids, lpp, pstride, ps[i], ps[i].s0 == 0 ? 1 : 0,
                          ps[i].s0 == 0 ? osc : nullptr);
    LAUNCH_CHECK();
}

void ntt_inverse_from(const ckks_ctx* c, const u64* src, size_t src_pstride, u64* data, int nlimbs, const int* ids,
                      int lpp, size_t pstride, const u64* osc, u64 kres, int k_id) {
    if (nlimbs <= 0) return;
    if (pstride == 0) pstride = (size_t)lpp * c->n;
    const bool scaled = k_id >= 0 && kres != 1;
    CK_CHECK(nlimbs % lpp == 0, CKKS_EINVAL, "whole polynomials only");
    CK_CHECK(!scaled || (lpp == 1 && osc == nullptr && pstride == c->n), CKKS_EINVAL,
             "an integer factor needs one contiguous row per polynomial and no output scale table");
    if (c->logn == 16) {
        NttSrc io{src, src_pstride, 0, 0};
        if (scaled) {
            const u64 q = c->mod_of[k_id];
            io.ow = hostmath::mulmod(kres, hostmath::invmod((u64)c->n % q, q), q);
            io.owp = hostmath::shoup(io.ow, q);
        }
        launch_ntt_transform<true>(c, data, nlimbs, ids, lpp, pstride, nullptr, osc, io);
        LAUNCH_CHECK();
        return;
    }
    // the smaller rings: copy (and scale), then transform in place
    if (scaled) {
        ScalarVec sv;
        sv.v[0] = kres;
        sv.vp[0] = hostmath::shoup(kres, c->mod_of[k_id]);
        mul_scalar_v(c, src, sv, data, nlimbs, ids, 1, src_pstride);
    } else {
        CUDA_CHECK(cudaMemcpy2DAsync(data, pstride * 8, src, src_pstride * 8, (size_t)lpp * c->n * 8, nlimbs / lpp,
                                     cudaMemcpyDeviceToDevice, c->stream));
    }
    ntt_inverse(c, data, nlimbs, ids, lpp, pstride, osc);
}

void add(const ckks_ctx* c, const u64* a, const u64* b, u64* o, int nl, const int* ids, int lpp) {
    if (nl <= 0) return;
    { KTimer kt_(c, "add", 3.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_add, al16(a) && al16(b) && al16(o), nl, a, b, o, c->d_primes, ids, lpp, c->logn);
    }
    LAUNCH_CHECK();
}
void sub(const ckks_ctx* c, const u64* a, const u64* b, u64* o, int nl, const int* ids, int lpp) {
    if (nl <= 0) return;
    { KTimer kt_(c, "sub", 3.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_sub, al16(a) && al16(b) && al16(o), nl, a, b, o, c->d_primes, ids, lpp, c->logn);
    }
    LAUNCH_CHECK();
}
void neg(const ckks_ctx* c, const u64* a, u64* o, int nl, const int* ids, int lpp) {
    if (nl <= 0) return;
    { KTimer kt_(c, "neg", 2.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_neg, al16(a) && al16(o), nl, a, o, c->d_primes, ids, lpp, c->logn);
    }
    LAUNCH_CHECK();
}
void mul(const ckks_ctx* c, const u64* a, const u64* b, u64* o, int nl, const int* ids, int lpp, int bmod) {
    if (nl <= 0) return;
    { KTimer kt_(c, "mul", (bmod ? 2.0 + (double)bmod / nl : 3.0) * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_mul, al16(a) && al16(b) && al16(o), nl, a, b, o, c->d_primes, ids, lpp, c->logn, bmod);
    }
    LAUNCH_CHECK();
}
void tensor(const ckks_ctx* c, const u64* a, const u64* b, u64* d, u64* e, int nl, const int* ids, int nb,
            size_t ab_bstride, size_t d_bstride, size_t e_bstride) {
    if (nl <= 0 || nb <= 0) return;
    const bool vec = al16(a) && al16(b) && al16(d) && al16(e);
    dim3 grid = ewv_grid(c->n, nl, vec ? 2 : 1);
    grid.z = nb;
    { KTimer kt_(c, "tensor", 7.0 * (double)nl * nb * c->n * 8.0);
    if (vec)
        klaunch(c, k_tensor<2>, grid, EW_THREADS, 0, a, b, d, e, c->d_primes, ids, nl, c->logn, ab_bstride, d_bstride,
                e_bstride);
    else
        klaunch(c, k_tensor<1>, grid, EW_THREADS, 0, a, b, d, e, c->d_primes, ids, nl, c->logn, ab_bstride, d_bstride,
                e_bstride);
    }
    LAUNCH_CHECK();
}
void mul_acc(const ckks_ctx* c, const u64* a, const u64* b, u64* o, int nl, const int* ids, int lpp) {
    if (nl <= 0) return;
    { KTimer kt_(c, "mul_acc", 4.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_mul_acc, al16(a) && al16(b) && al16(o), nl, a, b, o, c->d_primes, ids, lpp, c->logn);
    }
    LAUNCH_CHECK();
}
void mul_scalar(const ckks_ctx* c, const u64* a, const u64* s, const u64* sp, u64* o, int nl, const int* ids,
                int lpp) {
    if (nl <= 0) return;
    { KTimer kt_(c, "mul_scalar", 2.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_mul_scalar, al16(a) && al16(o), nl, a, s, sp, o, c->d_primes, ids, lpp, c->logn);
    }
    LAUNCH_CHECK();
}
void mul_scalar_v(const ckks_ctx* c, const u64* a, const ScalarVec& sv, u64* o, int nl, const int* ids, int lpp,
                  size_t a_pstride) {
    if (nl <= 0) return;
    CK_CHECK(lpp <= ScalarVec::MAX, CKKS_EINVAL, "too many limbs for a by-value scalar vector");
    { KTimer kt_(c, "mul_scalar", 2.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_mul_scalar_v, al16(a) && al16(o) && a_pstride % 2 == 0, nl, a, sv, o, c->d_primes, ids, lpp,
               a_pstride, c->logn);
    }
    LAUNCH_CHECK();
}
void sub_mul2_scalar(const ckks_ctx* c, const u64* a, const u64* b, const ScalarVec& s1, const u64* s2,
                     const u64* s2p, u64* o, int nl, const int* ids, int lpp, size_t a_pstride) {
    if (nl <= 0) return;
    CK_CHECK(lpp <= ScalarVec::MAX, CKKS_EINVAL, "too many limbs for a by-value scalar vector");
    { KTimer kt_(c, "sub_mul_scalar", 3.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_sub_mul2_scalar, al16(a) && al16(b) && al16(o) && a_pstride % 2 == 0, nl, a, b, s1, s2, s2p, o,
               c->d_primes, ids, lpp, a_pstride, c->logn);
    }
    LAUNCH_CHECK();
}
void lincomb(const ckks_ctx* c, const LinComb& t, u64* o, int nl, const int* ids, int lpp) {
    if (nl <= 0) return;
    CK_CHECK(t.n >= 1 && t.n <= LinComb::MAX && lpp <= LinComb::MAXL, CKKS_EINVAL,
             "1..16 terms over at most 40 limbs per linear combination");
    bool vec = al16(o);
    for (int i = 0; i < t.n; ++i) vec = vec && al16(t.a[i]);
    { KTimer kt_(c, "lincomb", (t.n + 1.0) * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_lincomb, vec, nl, t, o, c->d_primes, ids, lpp, c->logn);
    }
    LAUNCH_CHECK();
}
void add_scalar_v(const ckks_ctx* c, u64* a, const ScalarVec& sv, int nl, const int* ids, int lpp,
                  size_t a_pstride) {
    if (nl <= 0) return;
    CK_CHECK(lpp <= ScalarVec::MAX, CKKS_EINVAL, "too many limbs for a by-value scalar vector");
    { KTimer kt_(c, "add_scalar", 2.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_add_scalar_v, al16(a) && a_pstride % 2 == 0, nl, a, sv, c->d_primes, ids, lpp, c->logn, a_pstride);
    }
    LAUNCH_CHECK();
}
void add_const_term(const ckks_ctx* c, u64* a, const u64* v, int nl, const int* ids) {
    if (nl <= 0) return;
    { KTimer kt_(c, "add_scalar", 2.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_add_scalar, al16(a), nl, a, v, c->d_primes, ids, c->logn);
    }
    LAUNCH_CHECK();
}
void small_to_rns(const ckks_ctx* c, const int64_t* v, u64* o, int nl, const int* ids) {
    if (nl <= 0) return;
    { KTimer kt_(c, "small_to_rns", (nl + 1.0) * c->n * 8.0);
    klaunch(c, k_small_to_rns, ew_grid(c->n, nl), EW_THREADS, 0, v, o, c->d_primes, ids, c->logn);
    }
    LAUNCH_CHECK();
}
void automorph(const ckks_ctx* c, const u64* a, u64* o, int nl, u64 g) {
    if (nl <= 0) return;
    { KTimer kt_(c, "automorph", 2.0 * (double)nl * c->n * 8.0);
    klaunch(c, k_automorph, ew_grid(c->n, nl), EW_THREADS, 0, a, o, g, c->logn);
    }
    LAUNCH_CHECK();
}
void automorph_acc(const ckks_ctx* c, const u64* a, u64* o, int nl, u64 g, const u64* s, const u64* sp,
                   const int* ids, int lpp) {
    if (nl <= 0) return;
    { KTimer kt_(c, "automorph_acc", 3.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_automorph_acc, al16(o), nl, a, o, g, s, sp, c->d_primes, ids, lpp, c->logn);
    }
    LAUNCH_CHECK();
}
void imult(const ckks_ctx* c, const u64* a, u64* o, int nl, const int* ids, int lpp) {
    if (nl <= 0) return;
    { KTimer kt_(c, "imult", 2.0 * (double)nl * c->n * 8.0);
    klaunch(c, k_imult, ew_grid(c->n, nl), EW_THREADS, 0, a, o, c->d_primes, ids, lpp, c->logn);
    }
    LAUNCH_CHECK();
}
void lift_centred(const ckks_ctx* c, const u64* src, int src_id, u64* o, int nl, const int* ids, int lpp,
                  size_t src_pstride) {
    if (nl <= 0) return;
    if (lpp <= 0) lpp = nl;
    { KTimer kt_(c, "lift_centred", (nl + 1.0) * c->n * 8.0);
    EWV_LAUNCH(k_lift_centred, al16(src) && al16(o) && src_pstride % 2 == 0, nl, src, c->mod_of[src_id], o,
               c->d_primes, ids, lpp, src_pstride, c->logn);
    }
    LAUNCH_CHECK();
}
void sub_mul_scalar(const ckks_ctx* c, const u64* a, const u64* b, const u64* s, const u64* sp, u64* o, int nl,
                    const int* ids, int lpp, size_t a_pstride) {
    if (nl <= 0) return;
    { KTimer kt_(c, "sub_mul_scalar", 3.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_sub_mul_scalar, al16(a) && al16(b) && al16(o) && a_pstride % 2 == 0, nl, a, b, s, sp, o, c->d_primes,
               ids, lpp, a_pstride, c->logn);
    }
    LAUNCH_CHECK();
}
void base_convert(const ckks_ctx* c, const ConvTab& t, const u64* in, size_t in_stride, u64* out,
                  size_t out_stride, int npoly, size_t in_pstride, size_t out_pstride, bool prescaled) {
    CK_CHECK(in_stride == (size_t)c->n && out_stride == (size_t)c->n, CKKS_EINVAL, "limbs must be contiguous");
    ConvJobs J;
    J.n = 0;
    add_conv_job(J, t, in, out, in_pstride, out_pstride, prescaled);
    base_convert_jobs(c, J, npoly);
}

void add_conv_job(ConvJobs& J, const ConvTab& t, const u64* in, u64* out, size_t in_pstride, size_t out_pstride,
                  bool prescaled) {
    CK_CHECK(J.n < ConvJobs::MAX, CKKS_EINVAL, "too many base-conversion jobs");
    CK_CHECK(t.nin <= MAX_CONV_IN, CKKS_EINVAL, "base conversion with more than 16 input limbs");
    ConvJob& j = J.job[J.n++];
    j.in = in;
    j.out = out;
    j.in_ids = t.d_in_ids;
    j.out_ids = t.d_out_ids;
    j.out_rows = t.d_out_ids + t.nout;
    j.qinv = t.d_qhat_inv;
    j.qmod = t.d_qhat_mod;
    j.inv_q = t.d_inv_q;
    j.corr = t.d_corr;
    j.nin = t.nin;
    j.nout = t.nout;
    j.ngroups = (t.nout + CONV_OUT - 1) / CONV_OUT;
    j.in_pstride = in_pstride;
    j.out_pstride = out_pstride;
    j.prescaled = prescaled;
    j.tcb = t.d_tcb;
    j.tcr = t.d_tcr;
    j.tc_nin2 = t.tc_nin2;
    j.tc_S = t.tc_S;
}

template <int MAXIN, bool SPLIT>
static void launch_base_convert(const ckks_ctx* c, const ConvJobs& J, dim3 grid, int mc) {
    switch (mc) {
        case 4: klaunch(c, k_base_convert<MAXIN, SPLIT, 4>, grid, 256, 0, J, c->d_primes, c->logn); break;
        case 5: klaunch(c, k_base_convert<MAXIN, SPLIT, 5>, grid, 256, 0, J, c->d_primes, c->logn); break;
        case 6: klaunch(c, k_base_convert<MAXIN, SPLIT, 6>, grid, 256, 0, J, c->d_primes, c->logn); break;
        case 7: klaunch(c, k_base_convert<MAXIN, SPLIT, 7>, grid, 256, 0, J, c->d_primes, c->logn); break;
        default: klaunch(c, k_base_convert<MAXIN, SPLIT, 8>, grid, 256, 0, J, c->d_primes, c->logn); break;
    }
}

// Outputs per group MC in 4..8: the one with the fewest idle output slots over the launch's
// jobs (sum of ceil(nout / MC) MC - nout); on ties 6, 5, 4 (4 resident CTAs per SM) before
// 8, 7 (3 per SM).
void base_convert_jobs(const ckks_ctx* c, const ConvJobs& J0, int npoly) {
    if (conv_tc_eligible(c, J0)) {
        base_convert_tc_jobs(c, J0, npoly);
        LAUNCH_CHECK();
        return;
    }
    int best_mc = CONV_OUT, best_slots = -1;
    for (int mc : {6, 5, 4, 8, 7}) {
        int slots = 0;
        for (int i = 0; i < J0.n; ++i) slots += (J0.job[i].nout + mc - 1) / mc * mc;
        if (best_slots < 0 || slots < best_slots) {
            best_slots = slots;
            best_mc = mc;
        }
    }
    ConvJobs J = J0;
    int groups = 0;
    double bytes = 0;
    for (int i = 0; i < J.n; ++i) {
        J.job[i].ngroups = (J.job[i].nout + best_mc - 1) / best_mc;
        groups += J.job[i].ngroups;
        bytes += (double)npoly * (J.job[i].nin + J.job[i].nout) * c->n * 8.0;
    }
    if (groups == 0) return;
    int maxin = 0;
    for (int i = 0; i < J.n; ++i) maxin = std::max(maxin, J.job[i].nin);
    dim3 grid((c->n + 255) / 256, npoly, groups);
    { KTimer kt_(c, "base_convert", bytes);
    if (maxin <= 4)
        launch_base_convert<4, false>(c, J, grid, best_mc);
    else if (maxin <= 8 && c->mods_below_2_60)
        launch_base_convert<8, true>(c, J, grid, best_mc);
    else if (maxin <= 8)
        launch_base_convert<8, false>(c, J, grid, best_mc);
    else
        launch_base_convert<MAX_CONV_IN, false>(c, J, grid, best_mc);
    }
    LAUNCH_CHECK();
}

template <bool ACC, int V>
static void launch_ks_inner(const ckks_ctx* c, const u64* D, int ndig, int next, const int* ext_ids, const u64* kb,
                            const u64* ka, u64* ob, u64* oa, u64 g, const u64* x0, const u64* x1, int x0rows,
                            const u64* s0, const u64* s0p, const KsBatch& bt) {
    dim3 grid = ewv_grid(c->n, next, V);
    grid.x *= bt.nb;
    const size_t ks = (size_t)c->nall << c->logn;
    switch (ndig) {
        case 1:
            klaunch(c, k_ks_inner_d<ACC, V, 1>, grid, EW_THREADS, 0, D, next, ext_ids, kb, ka, ob, oa, c->d_primes,
                    c->logn, g, ks, x0, x1, x0rows, s0, s0p, bt);
            break;
        case 2:
            klaunch(c, k_ks_inner_d<ACC, V, 2>, grid, EW_THREADS, 0, D, next, ext_ids, kb, ka, ob, oa, c->d_primes,
                    c->logn, g, ks, x0, x1, x0rows, s0, s0p, bt);
            break;
        case 3:
            klaunch(c, k_ks_inner_d<ACC, V, 3>, grid, EW_THREADS, 0, D, next, ext_ids, kb, ka, ob, oa, c->d_primes,
                    c->logn, g, ks, x0, x1, x0rows, s0, s0p, bt);
            break;
        case 4:
            klaunch(c, k_ks_inner_d<ACC, V, 4>, grid, EW_THREADS, 0, D, next, ext_ids, kb, ka, ob, oa, c->d_primes,
                    c->logn, g, ks, x0, x1, x0rows, s0, s0p, bt);
            break;
        default:
            klaunch(c, k_ks_inner<ACC, V>, grid, EW_THREADS, 0, D, ndig, next, ext_ids, kb, ka, ob, oa, c->d_primes,
                    c->logn, g, ks);
            break;
    }
}

void ks_inner(const ckks_ctx* c, const u64* D, int ndig, int next, const int* ext_ids, const u64* kb,
              const u64* ka, u64* ob, u64* oa, u64 g, bool accumulate, const u64* x0, int x0rows, const u64* s,
              const u64* sp, const u64* x1, const KsBatch& bt) {
    CK_CHECK(bt.nb >= 1 && (bt.nb == 1 || ndig <= 4), CKKS_EINVAL, "batched key switching needs at most 4 digits");
    const bool vec = al16(kb) && al16(ka) && al16(ob) && al16(oa);
    const bool fuse = x0 && x0rows > 0 && ndig <= 4;   // the generic kernel adds x0, x1 in further passes
    {
        // algorithmic bytes: the key once for the whole batch, per ciphertext its digits, outputs
        // (read too when accumulating) and the x0 / x1 rows
        const double extra = fuse ? (double)x0rows * (x1 ? 2.0 : 1.0) / next : 0.0;
        KTimer kt_(c, "ks_inner",
                   (2.0 * ndig + bt.nb * (ndig + (accumulate ? 4.0 : 2.0) + extra)) * next * c->n * 8.0);
        const u64* fx = fuse ? x0 : nullptr;
        const u64* fy = fuse ? x1 : nullptr;
        if (accumulate) {
            if (vec)
                launch_ks_inner<true, 2>(c, D, ndig, next, ext_ids, kb, ka, ob, oa, g, fx, fy, x0rows, s, sp, bt);
            else
                launch_ks_inner<true, 1>(c, D, ndig, next, ext_ids, kb, ka, ob, oa, g, fx, fy, x0rows, s, sp, bt);
        } else {
            if (vec)
                launch_ks_inner<false, 2>(c, D, ndig, next, ext_ids, kb, ka, ob, oa, g, fx, fy, x0rows, s, sp, bt);
            else
                launch_ks_inner<false, 1>(c, D, ndig, next, ext_ids, kb, ka, ob, oa, g, fx, fy, x0rows, s, sp, bt);
        }
    }
    LAUNCH_CHECK();
    if (x0 && x0rows > 0 && !fuse) {
        automorph_acc(c, x0, ob, x0rows, g, s, sp, ext_ids, x0rows);
        if (x1) automorph_acc(c, x1, oa, x0rows, g, s, sp, ext_ids, x0rows);
    }
}
void mul_scalar_acc(const ckks_ctx* c, const u64* a, const u64* s, const u64* sp, u64* o, int nl, const int* ids,
                    int lpp, size_t o_pstride) {
    if (nl <= 0) return;
    { KTimer kt_(c, "mul_scalar_acc", 3.0 * (double)nl * c->n * 8.0);
    EWV_LAUNCH(k_mul_scalar_acc, al16(a) && al16(o) && o_pstride % 2 == 0, nl, a, s, sp, o, c->d_primes, ids, lpp,
               c->logn, o_pstride);
    }
    LAUNCH_CHECK();
}
void sample_uniform(const ckks_ctx* c, u64* o, int nl, const int* ids, u64 key) {
    if (nl <= 0) return;
    { KTimer kt_(c, "sample_uniform", (double)nl * c->n * 8.0);
    klaunch(c, k_sample_uniform, ew_grid(c->n, nl), EW_THREADS, 0, o, c->d_primes, ids, c->logn, key);
    }
    LAUNCH_CHECK();
}
void sample_small(const ckks_ctx* c, int64_t* o, u64 key, int kind) {
    { KTimer kt_(c, "sample_small", c->n * 8.0);
    klaunch(c, k_sample_small, ew_grid(c->n, 1), EW_THREADS, 0, o, c->logn, key, kind, c->d_gauss);
    }
    LAUNCH_CHECK();
}

}  // namespace kern
