// Fast base conversion on the tensor cores (tcgen05 MMA, tensor memory, bulk copies; sm_103a).
//
// The conversion of the hybrid key switch (ModUp of each digit, ModDown, ModDown fused with
// the rescale) computes, for every coefficient j,
//     y_m(j) = sum_i xh_i(j) c_{m,i}  mod p_m,     xh_i = [x_i qhat_i^{-1}]_{q_i},
// a matrix product of the N x nin input words with the nin x nout table.  64-bit words do not
// fit a tensor-core operand, so both sides are cut into 8-bit chunks:
//     xh_i = sum_a x_{i,a} 2^(8a),
//     e_{m,i,a} = c_{m,i} 2^(8a) mod p_m = sum_b e_{m,i,a,b} 2^(8b)      (a, b = 0..7),
// and then
//     y_m = sum_b 2^(8b) D_{m,b}  (mod p_m),    D_{m,b} = sum_{i,a} x_{i,a} e_{m,i,a,b}.
// D is an ordinary matrix product with K = 8 nin and 8 columns per output.  Every operand is
// an integer in [0, 255] (exact in FP16) and every D is a sum of at most 8 * 16 products
// below 2^16, so it stays below 2^23.  The accumulators start at 2^23 instead of 0: every
// partial sum is then an integer in [2^23, 2^24), exact in FP32 with a fixed exponent, and
// the final word's low 23 bits are D itself, from which the value of sum_b 2^(8b) D_{m,b} is
// assembled and reduced mod p_m (with, for an exact table, the
// rounded correction v (Q mod p_m) of the integer-pipe kernel, Halevi-Polyakov-Shoup 2019).
// Every output goes to a forward NTT.  For N = 2^16 the words are left congruent but below 4p
// (the radix-16 transform's lazy butterflies take such inputs and end canonical); otherwise they
// are the canonical residues.  Either way the transformed words equal the integer-pipe
// kernel's.
//
// A CTA takes 128 coefficients per tile (MMA M = 128, one TMEM lane per coefficient) for one
// output group of S <= 16 outputs (N = 8 S <= 128 TMEM columns, four CTAs per SM fill the
// 512 columns) and walks over `tiles` consecutive tiles.  The group's B image (the chunked
// table, precomputed on the host in the MMA's shared-memory layout) comes in by one bulk
// copy; each thread cuts its coefficient's input words into the A tile, one elected thread
// issues the K / 16 MMAs and commits them to an mbarrier, and every thread then reads its
// TMEM lane and writes its outputs (coalesced across the warp).  The next tile's inputs are
// loaded while the MMAs and the epilogue of the current tile run.
//
// Shared-memory operand layout (no swizzle, K-major): 8 x 8 FP16 core matrices of 128
// contiguous bytes; core (r, k) of a tile at (r * K/8 + k) * 128 bytes, so the leading
// (K-direction) byte offset is 128 and the stride (8-row) byte offset K/8 * 128.  Row j of
// core (r, i) holds the 8 chunks of input word i of coefficient 8 r + j: one 16-byte store.
#include "launch.cuh"

namespace {

__device__ unsigned g_tc_faults;   // bounded waits that ran out (read and cleared by the host)
// test hook: nonzero withholds the MMAs and their commit, so that every tile's bounded wait on
// the MMA barrier runs out (the path a lost completion would take); set only by tests
__device__ unsigned g_tc_withhold;

constexpr int TC_M = 128;               // coefficients per tile: MMA M, TMEM lanes
constexpr int TC_MAXIN = 16;
constexpr int TC_MAXS = 16;             // outputs per group: 8 S <= 128 TMEM columns
constexpr int TC_CTAS_PER_SM = 4;       // 4 x 128 columns = the SM's tensor memory
// dynamic shared memory per CTA is at least this much, so that no more than four CTAs are
// resident on an SM and a tensor-memory allocation never waits on a fifth
constexpr unsigned TC_SMEM_FLOOR = 46u * 1024u;
constexpr long long TC_WAIT_CYCLES = 1ll << 31;   // ~1 s at 2 GHz

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// the thread is suspended until the phase completes or about 0.5 ms pass (a hint, in ns)
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(500000u)
        : "memory");
    return done != 0;
}
// wait for the phase of the given parity to complete; false after ~1 s (the caller records
// the fault and leaves)
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > TC_WAIT_CYCLES) return false;
    return true;
}
// global -> shared bulk copy completing on an mbarrier (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// generic-proxy writes to shared memory made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(unsigned dst_smem, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: start address, leading / stride byte offsets (all >> 4),
// descriptor version 1 (bit 46), no swizzle, base offset 0
__device__ __forceinline__ u64 smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (u64)((addr & 0x3FFFFu) >> 4) | ((u64)((lbo >> 4) & 0x3FFFu) << 16) |
           ((u64)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B FP16 (bits
// 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ unsigned idesc_f16_f32(int m, int n) {
    return (1u << 4) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}
// D[tmem] (+)= A[smem] B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_f16(unsigned dtmem, u64 adesc, u64 bdesc, unsigned idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the mbarrier completes one arrival when every MMA this thread issued so far has finished
__device__ __forceinline__ void mma_commit(unsigned bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane; the registers are passed through
// the wait so that nothing reads them before the load has completed
__device__ __forceinline__ void tmem_ld16(unsigned taddr, unsigned (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane set to v
__device__ __forceinline__ void tmem_st16(unsigned taddr, unsigned v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1};" ::"r"(taddr),
        "r"(v)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// the 8 bytes of x as FP16 values, byte a in half a: each half is first 0x64bb (the FP16
// number 1024 + bb), then 1024 is subtracted exactly
__device__ __forceinline__ uint4 chunks_f16(u64 x) {
    const unsigned lo = (unsigned)x, hi = (unsigned)(x >> 32), k = 0x64006400u;
    uint4 h;
    h.x = __byte_perm(lo, 0x64646464u, 0x4140);
    h.y = __byte_perm(lo, 0x64646464u, 0x4342);
    h.z = __byte_perm(hi, 0x64646464u, 0x4140);
    h.w = __byte_perm(hi, 0x64646464u, 0x4342);
    asm("sub.rn.f16x2 %0, %0, %4;\n\t"
        "sub.rn.f16x2 %1, %1, %4;\n\t"
        "sub.rn.f16x2 %2, %2, %4;\n\t"
        "sub.rn.f16x2 %3, %3, %4;"
        : "+r"(h.x), "+r"(h.y), "+r"(h.z), "+r"(h.w)
        : "r"(k));
    return h;
}

// y = sum_b 2^(8b) D_b mod p from the FP32 words w_b = 2^23 + D_b (bit patterns
// 0x4B000000 + D_b, D_b < 2^23; the accumulators start at 2^23): lo = D_0 + 2^8 D_1 + 2^16 D_2 < 2^39 < p and
// hi = D_3 + ... + 2^32 D_7 < 2^56, y = lo + hi 2^24 mod p with one lazy Shoup product by
// 2^24 (< p; companion r24p = floor(2^88 / p)); the result lies in [0, 3p), not reduced
__device__ __forceinline__ u64 chunk_reduce_lazy(const unsigned* w, u64 p, u64 r24p) {
    constexpr u64 OFF_LO = 0x4B000000ull * 0x010101ull, OFF_HI = 0x4B000000ull * 0x0101010101ull;
    const u64 lo = (u64)w[0] + (u64)w[1] * 256u + (u64)w[2] * 65536u - OFF_LO;
    const u64 hi = (u64)w[3] + (u64)w[4] * 256u + (u64)w[5] * 65536u + (u64)w[6] * 16777216u +
                   ((u64)w[7] << 32) - OFF_HI;
    return lo + ((hi << 24) - __umul64hi(hi, r24p) * p);   // lo + [0, 2p) < 3p
}

// TPR threads per coefficient row (CTA = 128 TPR threads): thread (r, h) writes the chunks of
// the inputs i = h (mod TPR) of row r and finishes the output pairs p = h (mod TPR) of row r;
// warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31, the rows of its threads.  With
// TPR > 1 an exact table's rounding term needs all of a row's xh_i: they go through shared
// memory ([nin][128] words after the B image) and every thread of the row sums them in order.
// EXACT / PRE: every job of the launch has an exact table / prescaled inputs.  The
// accumulators of a tile are set to 2^23 before its first MMA, so that each holds 2^23 + D
// (exact: below 2^24) and its bit pattern exposes D directly.
template <int MAXIN, int TPR, bool EXACT, bool PRE, bool LAZY>
__global__ void __launch_bounds__(TC_M * TPR, TC_CTAS_PER_SM)
    k_base_convert_tc(kern::ConvJobs J, const DevPrime* __restrict__ P, int logn, int tiles) {
    constexpr bool lazy = LAZY;
    griddep_entry();
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) u64 s_bar[2];   // [0]: B image landed, [1]: MMAs of the tile done
    __shared__ unsigned s_taddr;
    __shared__ u64 s_qi[TC_MAXIN], s_qinv[TC_MAXIN], s_qinvp[TC_MAXIN];
    __shared__ u64 s_invm[TC_MAXIN];
    __shared__ int s_invs[TC_MAXIN];
    __shared__ u64 s_p[TC_MAXS], s_r24p[TC_MAXS], s_corr[TC_MAXS], s_corrp[TC_MAXS];
    __shared__ int s_row[TC_MAXS];

    int z = blockIdx.z, jb = 0;
    while (jb < J.n - 1 && z >= J.job[jb].ngroups) {
        z -= J.job[jb].ngroups;
        ++jb;
    }
    const kern::ConvJob& job = J.job[jb];
    const int nin = job.nin, nin2 = job.tc_nin2, S = job.tc_S;
    const int m0 = z * S;
    const int mcount = min(S, job.nout - m0);
    constexpr bool exact = EXACT;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (TC_M - 1), h = tid / TC_M;
    unsigned ncols = 32;
    while (ncols < 8u * S) ncols <<= 1;
    const unsigned sbo = (unsigned)nin2 * 128u;   // bytes per 8-row group of A and of B
    unsigned char* sA = tc_smem;
    unsigned char* sB = tc_smem + TC_M * nin2 * 16;
    u64* xs = reinterpret_cast<u64*>(sB + S * sbo);
    const unsigned bytesB = (unsigned)S * sbo;

    if (tid < nin) {
        s_qi[tid] = P[job.in_ids[tid]].m.q;
        s_qinv[tid] = job.qinv[tid];
        s_qinvp[tid] = job.qinv[nin + tid];
        s_invm[tid] = exact ? job.inv_q[tid] : 0;
        s_invs[tid] = exact ? (int)job.inv_q[nin + tid] : 64;
    }
    if (tid < mcount) {
        s_p[tid] = P[job.out_ids[m0 + tid]].m.q;
        s_r24p[tid] = job.tcr[m0 + tid];
        s_row[tid] = job.out_rows[m0 + tid];
        s_corr[tid] = exact ? job.corr[m0 + tid] : 0;
        s_corrp[tid] = exact ? job.corr[job.nout + m0 + tid] : 0;
    }
    const unsigned barB = smem_u32(&s_bar[0]), barM = smem_u32(&s_bar[1]);
    if (tid == 0) {
        mbar_init(barB, 1);
        mbar_init(barM, 1);
        mbar_init_fence();
    }
    __syncwarp();
    if (warp == 0) {
        tmem_alloc(smem_u32(&s_taddr), ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned taddr = s_taddr;
    if (tid == 0) {
        mbar_expect_tx(barB, bytesB);
        bulk_g2s(smem_u32(sB), job.tcb + (size_t)m0 * nin2 * 64, bytesB, barB);
    }

    const size_t n = (size_t)1 << logn;
    const u64* in = job.in + blockIdx.y * job.in_pstride;
    u64* out = job.out + blockIdx.y * job.out_pstride;
    const int ntiles = (int)(n / TC_M);
    const int t0 = blockIdx.x * tiles, t1 = min(ntiles, t0 + tiles);
    const unsigned idesc = idesc_f16_f32(TC_M, 8 * S);
    const unsigned aaddr = smem_u32(sA), baddr = smem_u32(sB);
    const unsigned tlane = taddr + ((unsigned)((warp & 3) * 32) << 16);
    unsigned char* arow = sA + (row >> 3) * sbo + (row & 7) * 16;
    bool ok = true, b_ready = false;
    unsigned phase = 0;

    constexpr int NX = MAXIN / TPR;   // this thread's inputs: i = k TPR + h
    u64 x[NX];
#pragma unroll
    for (int k = 0; k < NX; ++k)
        if (k * TPR + h < nin && t0 < t1) x[k] = in[(size_t)(k * TPR + h) * n + (size_t)t0 * TC_M + row];
    for (int t = t0; t < t1; ++t) {
        const size_t j = (size_t)t * TC_M + row;
        u64 f = 0;
#pragma unroll
        for (int k = 0; k < NX; ++k) {
            const int i = k * TPR + h;
            if (i < nin) {
                const u64 xh = PRE ? x[k] : mul_shoup(x[k], s_qinv[i], s_qinvp[i], s_qi[i]);
                if (exact) {
                    if (TPR == 1) f += conv_round_term(xh, s_invm[i], s_invs[i]);
                    else xs[i * TC_M + row] = xh;
                }
                *reinterpret_cast<uint4*>(arow + i * 128) = chunks_f16(xh);
            }
        }
        if (nin < nin2 && nin % TPR == h) *reinterpret_cast<uint4*>(arow + nin * 128) = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int k = 0; k < 8 / TPR; ++k) {
            const int p = h + k * TPR;
            if (p >= S / 2) break;
            tmem_st16(tlane + 16u * p, 0x4B000000u);
        }
        tmem_wait_st();
        tc_fence_before();
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            if (!b_ready) {
                b_ready = true;
                if (!mbar_wait(barB, 0)) ok = false;
            }
            tc_fence_after();
            if (ok && !*(volatile unsigned*)&g_tc_withhold) {
                for (int s = 0; s < nin2 / 2; ++s)
                    mma_f16(taddr, smem_desc(aaddr + 256u * s, 128u, sbo), smem_desc(baddr + 256u * s, 128u, sbo),
                            idesc, 1);
                mma_commit(barM);
            }
        }
        __syncwarp();
        if (TPR > 1 && exact) {
            for (int i = 0; i < nin; ++i) f += conv_round_term(xs[i * TC_M + row], s_invm[i], s_invs[i]);
        }
        const u64 v = exact ? conv_round_finish(f) : 0;
        // the next tile's inputs are in flight while the MMAs and this tile's epilogue run
        if (t + 1 < t1) {
#pragma unroll
            for (int k = 0; k < NX; ++k)
                if (k * TPR + h < nin) x[k] = in[(size_t)(k * TPR + h) * n + j + TC_M];
        }
        if (!mbar_wait(barM, phase)) ok = false;
        phase ^= 1u;
        tc_fence_after();
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8 / TPR; ++k) {
            const int p = h + k * TPR;
            if (p >= S / 2) break;
            unsigned r[16];
            tmem_ld16(tlane + 16u * p, r);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int m = 2 * p + e;
                if (m >= mcount) continue;   // only the last group of a table can be short
                const u64 pm = s_p[m];
                u64 y = chunk_reduce_lazy(r + 8 * e, pm, s_r24p[m]);
                if (lazy) {
                    // the forward NTT of N = 2^16 takes inputs below 4p
                    if (exact) y += mul_shoup(v, s_corr[m], s_corrp[m], pm);
                } else {
                    if (y >= 2 * pm) y -= 2 * pm;
                    if (y >= pm) y -= pm;
                    if (exact) y = add_mod(y, mul_shoup(v, s_corr[m], s_corrp[m], pm), pm);
                }
                out[(size_t)s_row[m] * n + j] = y;
            }
        }
        tc_fence_before();
        if (__syncthreads_or(!ok)) break;
    }
    // the B image must have landed before the CTA's shared memory goes away
    if (tid == 0 && !b_ready && !mbar_wait(barB, 0)) ok = false;
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(taddr, ncols);
    }
    if (!ok) atomicAdd(&g_tc_faults, 1u);
}

}  // namespace

namespace kern {

// FP16 bit pattern of an integer in [0, 255]
static unsigned short half_bits(unsigned v) {
    if (v == 0) return 0;
    int e = 0;
    while ((v >> (e + 1)) != 0) ++e;
    return (unsigned short)(((unsigned)(e + 15) << 10) | ((v << (10 - e)) & 0x3FFu));
}

std::vector<unsigned short> conv_tc_image(const std::vector<u64>& qmod, const std::vector<u64>& pm, int nin, int nout,
                                          int& nin2, int& S, int& groups, std::vector<u64>& r24p) {
    // the epilogue needs every output modulus above 2^39 (see chunk_reduce) and below 2^62
    for (u64 p : pm)
        if (p <= (1ull << 39) || p >= (1ull << 62) || nin > TC_MAXIN) return {};
    r24p.resize(nout);
    for (int m = 0; m < nout; ++m) r24p[m] = (u64)(((unsigned __int128)1 << 88) / pm[m]);
    nin2 = (nin + 1) & ~1;
    groups = (nout + TC_MAXS - 1) / TC_MAXS;
    S = (nout + groups - 1) / groups;
    S += S & 1;
    std::vector<unsigned short> img((size_t)groups * S * nin2 * 64, 0);
    for (int m = 0; m < nout; ++m) {
        const u64 p = pm[m];
        for (int i = 0; i < nin; ++i) {
            u64 e = qmod[(size_t)m * nin + i] % p;
            for (int a = 0; a < 8; ++a) {
                for (int b = 0; b < 8; ++b)
                    img[(((size_t)m * nin2 + i) * 8 + b) * 8 + a] = half_bits((unsigned)((e >> (8 * b)) & 0xFF));
                e = hostmath::mulmod(e, 256 % p, p);
            }
        }
    }
    return img;
}

bool conv_tc_eligible(const ckks_ctx* c, const ConvJobs& J) {
    if (!c->conv_tc || c->n < (size_t)TC_M) return false;
    for (int i = 0; i < J.n; ++i)
        if (J.job[i].tcb == nullptr || J.job[i].nin > TC_MAXIN) return false;
    return J.n > 0;
}

template <int MAXIN, int TPR, bool EXACT, bool PRE, bool LAZY>
static void launch_tc(const ckks_ctx* c, const ConvJobs& J, dim3 grid, unsigned smem, int per) {
    // the attribute is set once per device for the largest operand tiles (K = 128, S = 16)
    constexpr int SMEM_MAX = TC_M * TC_MAXIN * 16 + TC_MAXS * TC_MAXIN * 128 + TC_M * TC_MAXIN * 8;
    static std::atomic<unsigned> done{0};
    allow_dynamic_smem((const void*)k_base_convert_tc<MAXIN, TPR, EXACT, PRE, LAZY>, SMEM_MAX, done);
    klaunch(c, k_base_convert_tc<MAXIN, TPR, EXACT, PRE, LAZY>, grid, TC_M * TPR, smem, J, c->d_primes, c->logn, per);
}

template <int MAXIN, int TPR, bool LAZY>
static void launch_tc_flags(const ckks_ctx* c, const ConvJobs& J, dim3 grid, unsigned smem, int per, bool exact,
                            bool pre) {
    if (exact) {
        if (pre) launch_tc<MAXIN, TPR, true, true, LAZY>(c, J, grid, smem, per);
        else launch_tc<MAXIN, TPR, true, false, LAZY>(c, J, grid, smem, per);
    } else {
        if (pre) launch_tc<MAXIN, TPR, false, true, LAZY>(c, J, grid, smem, per);
        else launch_tc<MAXIN, TPR, false, false, LAZY>(c, J, grid, smem, per);
    }
}
// every conversion output goes to a forward NTT; for N = 2^16 its lazy butterflies take inputs
// below 4p, so the words are left in [0, 4p) there (canonical for the generic NTT)
template <int MAXIN, int TPR>
static void launch_tc_lazy(const ckks_ctx* c, const ConvJobs& J, dim3 grid, unsigned smem, int per, bool exact,
                           bool pre) {
    if (c->logn == 16) launch_tc_flags<MAXIN, TPR, true>(c, J, grid, smem, per, exact, pre);
    else launch_tc_flags<MAXIN, TPR, false>(c, J, grid, smem, per, exact, pre);
}

void base_convert_tc_jobs(const ckks_ctx* c, const ConvJobs& J0, int npoly) {
    // one launch per run of jobs that agree on the table kind and the input scaling
    for (int i = 1; i < J0.n; ++i) {
        if ((J0.job[i].inv_q != nullptr) != (J0.job[0].inv_q != nullptr) || J0.job[i].prescaled != J0.job[0].prescaled) {
            for (int k = 0; k < J0.n; ++k) {
                ConvJobs one;
                one.n = 1;
                one.job[0] = J0.job[k];
                base_convert_tc_jobs(c, one, npoly);
            }
            return;
        }
    }
    const bool exact = J0.n > 0 && J0.job[0].inv_q != nullptr, pre = J0.n > 0 && J0.job[0].prescaled;
    ConvJobs J = J0;
    int groups = 0, maxin = 0;
    unsigned smem = TC_SMEM_FLOOR;
    double bytes = 0;
    for (int i = 0; i < J.n; ++i) {
        ConvJob& jb = J.job[i];
        jb.ngroups = (jb.nout + jb.tc_S - 1) / jb.tc_S;
        groups += jb.ngroups;
        maxin = std::max(maxin, jb.nin);
        smem = std::max(smem, (unsigned)(TC_M * jb.tc_nin2 * 16 + jb.tc_S * jb.tc_nin2 * 128 + TC_M * jb.tc_nin2 * 8));
        bytes += (double)npoly * (jb.nin + jb.nout) * c->n * 8.0;
    }
    if (groups == 0) return;
    int dev = 0, nsm = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // tiles per CTA: the fewest that keep the grid within one wave of resident CTAs
    const int ntiles = (int)(c->n / TC_M);
    const long long cols = (long long)npoly * groups;
    const long long slots = (long long)nsm * TC_CTAS_PER_SM;
    int per = (int)std::max(1LL, (ntiles * cols + slots - 1) / slots);
    per = std::min(per, ntiles);
    const dim3 grid((ntiles + per - 1) / per, npoly, groups);
    KTimer kt_(c, "base_convert", bytes);
    const bool two = c->conv_tc_tpr == 2;
    if (maxin <= 8) {
        if (two) launch_tc_lazy<8, 2>(c, J, grid, smem, per, exact, pre);
        else launch_tc_lazy<8, 1>(c, J, grid, smem, per, exact, pre);
    } else {
        if (two) launch_tc_lazy<16, 2>(c, J, grid, smem, per, exact, pre);
        else launch_tc_lazy<16, 1>(c, J, grid, smem, per, exact, pre);
    }
}

void set_tc_withhold(bool on) {
    const unsigned v = on ? 1u : 0u;
    CUDA_CHECK(cudaMemcpyToSymbol(g_tc_withhold, &v, sizeof(v)));
}

unsigned peek_device_faults() {
    unsigned v = 0;
    CUDA_CHECK(cudaMemcpyFromSymbol(&v, g_tc_faults, sizeof(v)));
    return v;
}

unsigned take_device_faults() {
    unsigned v = 0, zero = 0;
    CUDA_CHECK(cudaMemcpyFromSymbol(&v, g_tc_faults, sizeof(v)));
    if (v) CUDA_CHECK(cudaMemcpyToSymbol(g_tc_faults, &zero, sizeof(zero)));
    return v;
}

}  // namespace kern
