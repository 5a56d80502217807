// Internal declarations of the GB300 RNS-CKKS library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "ckks.h"
#include "modarith.cuh"

typedef std::complex<double> cplx;

// ------------------------------------------------------------------ errors --
struct CkksError {
    int code;
    std::string msg;
};
#define CK_THROW(code, msg) throw CkksError{(code), (msg)}
#define CK_CHECK(cond, code, msg) \
    do {                          \
        if (!(cond)) CK_THROW(code, msg); \
    } while (0)
#define CUDA_CHECK(x)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (x);                                                               \
        if (e_ != cudaSuccess)                                                              \
            CK_THROW(e_ == cudaErrorMemoryAllocation ? CKKS_ENOMEM : CKKS_ECUDA,            \
                     std::string(#x) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

// ------------------------------------------------------------ device data --
// Per-prime constants, indexed by global prime id (q_0..q_L, then p_0..p_{np-1}).
struct DevPrime {
    DevMod m;
    const ulonglong2* tw;    // (psi^rev(k), Shoup companion), k < N   (forward, Cooley-Tukey)
    const ulonglong2* itw;   // (psi^-rev(k), Shoup companion)          (inverse, Gentleman-Sande)
    u64 n_inv, n_inv_p;
    u64 r64, r64p;           // 2^64 mod q and its Shoup companion (128-bit lazy sums)
    u64 inv64;               // floor(2^64 / q): Shoup companion of 1, reduces any 64-bit word
};

// Base-conversion table: inputs (prime ids in_ids, count nin) -> outputs (out_ids, nout).
//   xhat_i = x_i * qhat_inv[i] mod q_i ; y_m = sum_i xhat_i * qhat_mod[m*nin + i] mod p_m
struct ConvTab {
    int nin = 0, nout = 0;
    std::vector<int> in_ids, out_ids;
    int* d_in_ids = nullptr;
    int* d_out_ids = nullptr;
    u64* d_qhat_inv = nullptr;   // [nin] and Shoup [nin]
    u64* d_qhat_mod = nullptr;   // [nout][nin] and Shoup [nout][nin]
    // exact (rounded) conversion only: the reciprocals 1/q_i = M_i 2^-(64 + b_i) (b_i = bitlen(q_i)
    // - 1, M_i = floor(2^(64 + b_i) / q_i) in [2^63, 2^64)) as [nin] M_i then [nin] shifts b_i + 6;
    // p_m - (prod q_i mod p_m) [nout] followed by its Shoup companions [nout]
    u64* d_inv_q = nullptr;
    u64* d_corr = nullptr;
    // N^{-1} qhat_i^{-1} mod q_i and its Shoup companion, [nin][2]: the factor an inverse NTT
    // ends with when its output feeds this conversion directly (prescaled inputs)
    u64* d_iscale = nullptr;
    // tensor-core form (kern::base_convert_jobs with ctx->conv_tc): the table split into 8-bit
    // chunks as FP16 operands in the shared-memory image of the MMA's B operand,
    // [outputs padded to tc_S tc_groups][tc_nin2][8 chunks b of the entry][8 chunks a of the
    // input word] = chunk b of (qhat_mod[m][i] 2^(8a) mod p_m); inputs padded to an even count
    // tc_nin2, outputs to tc_groups groups of tc_S (even, <= 16)
    unsigned short* d_tcb = nullptr;
    u64* d_tcr = nullptr;        // floor(2^88 / p_m) [nout]: Shoup companion of 2^24 mod p_m
    int tc_nin2 = 0, tc_S = 0, tc_groups = 0;
};

// A caller-provided device allocator (ckks_ctx_set_allocator); both null = the library's own
// stream-ordered pool (cudaMallocAsync on the device's default memory pool).
struct DevAlloc {
    ckks_alloc_fn alloc = nullptr;
    ckks_free_fn free = nullptr;
    void* user = nullptr;
};
// The allocator of the context whose C-ABI call is running on this thread (set by that call's
// guard, null outside calls).  DevBufs made during the call take their memory from it, except
// while their stream is being captured into a CUDA graph (graph memory must live as long as
// the graph, so it comes from the stream-ordered pool).
extern thread_local const DevAlloc* tl_alloc;

// Device buffer owned by RAII: stream-ordered allocation on the context's stream, from the
// caller's allocator when one is set (the buffer remembers which, and frees through it).
struct DevBuf {
    u64* ptr = nullptr;
    size_t words = 0;
    cudaStream_t stream = 0;
    DevAlloc al;          // non-null alloc: allocated by this caller allocator
    DevBuf() {}
    DevBuf(size_t w, cudaStream_t s);
    ~DevBuf();
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
    DevBuf& operator=(DevBuf&& o) noexcept;
    void reset();
};

struct ckks_ctx {
    ckks_params P;
    int logn = 0, n = 0, nq = 0, L = 0, alpha = 0, np = 0, nall = 0, n_circuit = 0;
    bool mods_below_2_60 = false;    // every modulus < 2^60 (enables the split base conversion)
    std::vector<u64> q, p, psi;      // psi indexed by prime id
    std::vector<u64> mod_of;         // modulus by prime id
    std::vector<double> delta;
    std::vector<DevMod> mods;        // by prime id
    uint64_t seed = 0;
    u64 gauss[39];
    cudaStream_t stream = 0;
    // side streams for independent work inside one operation (the giant steps of an HMatmul,
    // the leaves of a Chebyshev evaluation); created on first use
    static constexpr int NSIDE = 4;
    cudaStream_t side[NSIDE] = {};
    cudaEvent_t fork_ev = nullptr, side_ev[NSIDE] = {};
    bool side_streams_on = true;
    // independent products inside one operation (a generation of the Chebyshev power ladder)
    // run as one lockstep batch instead of side by side on side streams
    bool inner_batching = false;
    // base conversions on the tensor cores (tcgen05 MMA of 8-bit chunks, exact FP32 sums)
    // instead of 64-bit multiply-adds on the integer pipe; results are identical either way
    bool conv_tc = true;
    int conv_tc_tpr = 1;    // threads per coefficient row of the tensor-core conversion (1 or 2)
    DevAlloc alloc;       // caller allocator for the buffers of this context's calls
    // side streams are used only without a caller allocator: a stream-ordered caching
    // allocator (PyTorch's) reuses a freed block on the stream it was allocated on, so every
    // buffer must be used on that one stream
    bool use_side_streams() const { return side_streams_on && alloc.alloc == nullptr; }
    DevPrime* d_primes = nullptr;
    u64* d_tables = nullptr;
    u64* d_gauss = nullptr;
    int* d_iota = nullptr;                   // 0..nall-1
    u64* d_pinv = nullptr;                   // P^{-1} mod q_i [nq], Shoup [nq]
    u64* d_qlinv = nullptr;                  // q_l^{-1} mod q_i [nq][nq], Shoup [nq][nq]
    std::vector<u64> h_qlinv;                // host copy of the residues [nq][nq]
    u64* d_pqlinv = nullptr;                 // (P q_l)^{-1} mod q_i [nq][nq], Shoup [nq][nq]
    u64* d_pqlinv2 = nullptr;                // the same times 2 (products doubled in the tail)
    u64* d_pmod = nullptr;                   // P mod q_i [nq], Shoup [nq]
    std::vector<int*> d_ext_ids;             // per level: [0..l] + specials
    // per level: the rows of the raised digits that ModUp converts (offsets in limbs
    // from the start of [ndig][next][N]) and their prime ids, for one NTT launch
    std::vector<int*> d_modup_off, d_modup_pid;
    std::vector<int> modup_nrows;
    // per level: for each of the l + 1 rows of a ModUp input, N^{-1} qhat^{-1} of its digit's
    // conversion (Shoup pairs, [l+1][2]), the inverse NTT's final factor for prescaled inputs
    std::vector<u64*> d_modup_iscale;
    std::map<std::pair<int, int>, std::unique_ptr<ConvTab>> modup_tabs;  // (level, digit)
    std::map<int, std::unique_ptr<ConvTab>> moddown_tabs;               // level
    std::map<int, std::unique_ptr<ConvTab>> mdrs_tabs;                  // level: {q_l, P} -> Q_{l-1}
    std::string err;
    int ntt_choice[8] = {-1, -1, -1, -1, -1, -1, -1, -1};   // tuned NTT variant per limb-count class
    // eager kernels are launched with programmatic stream serialization: the next launch in
    // the stream is set up while this one drains, and waits for it before touching memory
    bool pdl = true;
    std::map<std::string, long> ops;   // op counters (PMult, HRot, keyswitch, ...)
    // measurement: kernel launch count and, when timing is on, CUDA events around launches
    mutable long long launches = 0;
    bool timing = false;
    struct Pending {
        const char* name;
        cudaEvent_t a, b;
        double bytes;
    };
    struct KStat {
        long long launches = 0;
        double ms = 0, bytes = 0;
    };
    mutable std::vector<Pending> pending;
    mutable std::vector<cudaEvent_t> event_pool;
    mutable std::map<std::string, KStat> kstats;   // name -> launches, ms, algorithmic bytes
    void collect_timing() const;

    std::vector<std::vector<int>> digits(int level) const;
    std::vector<int> ext_ids(int level) const;
    const ConvTab& modup_tab(int level, int d);
    const ConvTab& moddown_tab(int level);
    const ConvTab& mdrs_tab(int level);
    ~ckks_ctx();
};

// A ciphertext, or a batch of nb ciphertexts at the same level and scale that every operation
// processes in lockstep (one launch per kernel for the whole batch, keys and plaintexts read
// once per launch): [nb][2][level+1][N].
struct ckks_ct {
    ckks_ctx* ctx = nullptr;
    DevBuf buf;           // [nb][2][level+1][N]
    int level = -1;
    double scale = 1.0;
    int nb = 1;
    size_t cstride() const { return 2 * (size_t)(level + 1) * ctx->n; }   // words per ciphertext
    u64* c0(int t = 0) const { return buf.ptr + t * cstride(); }
    u64* c1(int t = 0) const { return c0(t) + (size_t)(level + 1) * ctx->n; }
};

struct ckks_pt {
    ckks_ctx* ctx = nullptr;
    DevBuf buf;           // [level+1][N] (ext: [level+1+np][N], Q rows then P rows), NTT domain
    int level = -1;
    double scale = 1.0;
    bool ext = false;     // also reduced modulo the special primes (BSGS diagonals)
};

struct SwitchKey {
    DevBuf b, a;          // [ndig][nall][N], NTT domain
    int ndig = 0;
};

struct ckks_keys {
    ckks_ctx* ctx = nullptr;
    std::vector<int64_t> s;          // secret coefficients
    DevBuf s_ntt;                    // [nall][N]
    DevBuf pk_b, pk_a;               // [nq][N]
    std::map<u64, std::unique_ptr<SwitchKey>> swk;   // 0 = relin, else Galois element
};

struct ckks_ptset {
    ckks_ctx* ctx = nullptr;
    int a0 = 0, step = 1, count = 1, B = 1, level = 0;
    double scale = 1.0;
    std::map<std::pair<int, int>, std::unique_ptr<ckks_pt>> pts;
    int G() const { return (count + B - 1) / B; }
};

struct ckks_boot {
    ckks_ctx* ctx = nullptr;
    ckks_boot_params bp;
    int two_l = 0, ell = 0, C = 0, l_drop = 0, l_em = 0, l_out = 0;
    long long c_drop = 0;
    double K_eff = 0, s_raise = 0, s_em = 0, s_mask = 0;
    std::vector<double> coeffs;
    std::vector<std::unique_ptr<ckks_ptset>> ctos, stoc;
    std::unique_ptr<ckks_ptset> decomp;   // stride 2: Alg. 2 decomposition before StoC1
    std::unique_ptr<ckks_pt> mask_re, mask_im;
    bool mask_im_zero = false;   // the Im half of every slice is padding: its mask is exactly 0
    // What each BSGS level's plan is built from (CtoS levels, the stride-2 decomposition, the
    // StoC1 levels, in evaluation order), so that it can be rebuilt with another baby-step count.
    struct Level {
        int kind = 0;                 // 0 CtoS, 1 decomposition, 2 StoC1
        int index = 0;                // position in ctos / stoc
        std::vector<int> strides;     // DFT stages of a CtoS / StoC1 level
        bool half = false;            // the last CtoS level carries the factor 1/2
        int a0 = 0, step = 0, count = 0, level = 0;
        double scale = 0;
    };
    std::vector<Level> levels;
};

// Scope object placed around one kernel launch: counts it and, if the context's
// timing flag is set, brackets it with CUDA events on the context's stream.
struct KTimer {
    const ckks_ctx* c;
    const char* name;
    double bytes;
    cudaEvent_t a = nullptr, b = nullptr;
    KTimer(const ckks_ctx* ctx, const char* nm, double algo_bytes);
    ~KTimer();
};

// Per-limb residues (and Shoup companions) passed to a kernel by value.
struct ScalarVec {
    static constexpr int MAX = 40;
    u64 v[MAX];
    u64 vp[MAX];
};

// ----------------------------------------------------------- kernel API --
// All launchers enqueue on ctx->stream.  `ids` are device arrays of prime ids
// (length lpp = limbs per polynomial); limb k of a multi-polynomial array uses ids[k % lpp].
namespace kern {
// pstride: words between consecutive polynomials of lpp limbs (0 = lpp * N, contiguous)
void ntt_forward(const ckks_ctx* c, u64* data, int nlimbs, const int* ids, int lpp, size_t pstride = 0);
// forward NTT of an arbitrary list of limbs: limb i at data + off[i] * N with prime ids[i] (N = 2^16);
// for nb copies of the list, copy t at data + t * bstride
void ntt_forward_list(const ckks_ctx* c, u64* data, int nlimbs, const int* off, const int* ids, int nb = 1,
                      size_t bstride = 0);
// The inner sums of up to MAXG giant steps in one pass over the baby rotations (two
// polynomials of nl limbs each; limb r has prime ids[r]):
// o[g] (+)= sum_b a[b] * p[g][b] (p[g][b] null: zero diagonal), accumulating into o[g] when
// bit g of acc is set.  Every baby rotation is read once for all the giant steps.
struct BsgsGiants {
    static constexpr int MAXB = 32, MAXG = 8;
    const u64* a[MAXB];
    const u64* p[MAXG][MAXB];
    u64* o[MAXG];
    int nb, ng;
    unsigned acc;
};
// A batch of nb ciphertexts sharing keys and plaintexts: ciphertext t's operands at + t dstr,
// + t ostr and + t xstr words (which operand each stride moves is stated per call)
struct KsBatch {
    int nb = 1;
    size_t dstr = 0, ostr = 0, xstr = 0;
};
// (bt: a batch of bt.nb ciphertexts, babies at a[b] + t dstr, outputs at o[g] + t ostr)
void bsgs_inner_giants(const ckks_ctx* c, const BsgsGiants& t, int nl, const int* ids, const KsBatch& bt);
// Baby rotations and giant-step inner sums in one pass, the babies never stored: for every
// extended limb e and word j, baby b = (sum_d D_d(sigma_b) kb_b,d, sum_d D_d(sigma_b) ka_b,d)
// + (P c0(sigma_b), 0) on the Q rows (b with kb null: the identity, (P c0, P c1) on the Q rows,
// 0 on the P rows), then o[g] (+)= sum_b baby_b p[g][b] as in bsgs_inner_giants.
struct BsgsFused {
    static constexpr int MAXB = 32, MAXG = 4;
    const u64* kb[MAXB];
    const u64* ka[MAXB];
    u64 gal[MAXB];
    const u64* p[MAXG][MAXB];
    u64* o[MAXG];
    int nb, ng, ndig;
    unsigned acc;
};
// D [ndig][next][N] raised digits of c1; c0, c1 [nl][N]; s, sp: P mod q_i and Shoup
// (bt: a batch of bt.nb ciphertexts, D at + t dstr, c0 and c1 at + t xstr, outputs at o[g] + t ostr)
void bsgs_fused(const ckks_ctx* c, const BsgsFused& t, const u64* D, const u64* c0, const u64* c1, int nl,
                int next, const int* ext_ids, const u64* s, const u64* sp, const KsBatch& bt);
// o = sum_t w_t a_t (mod q per limb) for up to MAX terms: the integer-weighted sum of a
// Chebyshev leaf in one pass.  Arrays of nl limbs, limb k with prime ids[k % lpp]; w[t][r]
// is the weight's residue for limb index r < lpp, wp[t][r] its Shoup companion (passed by
// value: about 10 KB of kernel parameters).
struct LinComb {
    static constexpr int MAX = 16, MAXL = 40;
    const u64* a[MAX];
    u64 w[MAX][MAXL];
    u64 wp[MAX][MAXL];
    int n;
};
void lincomb(const ckks_ctx* c, const LinComb& t, u64* o, int nl, const int* ids, int lpp);
void autotune_ntt(ckks_ctx* c, int reps);
// (osc: per row r = k % lpp a Shoup pair (w, w') at osc[2r], osc[2r + 1] that replaces the final
// factor N^{-1}, e.g. N^{-1} qhat^{-1} for a base conversion that reads the output prescaled)
void ntt_inverse(const ckks_ctx* c, u64* data, int nlimbs, const int* ids, int lpp, size_t pstride = 0,
                 const u64* osc = nullptr);
// Inverse transform read out of place: row k of the input at src + (k / lpp) * src_pstride +
// (k % lpp) N, row k of the output at data + (k / lpp) * pstride + (k % lpp) N (pstride 0: lpp N);
// src is left unchanged; osc as in ntt_inverse.  k_id >= 0: one contiguous row per polynomial
// (lpp = 1, pstride N), all with the prime k_id, and the result is multiplied by kres (a residue
// mod that prime).  At N = 2^16 the first pass reads src and the last applies the factor;
// smaller rings copy (and scale) first.
void ntt_inverse_from(const ckks_ctx* c, const u64* src, size_t src_pstride, u64* data, int nlimbs, const int* ids,
                      int lpp, size_t pstride, const u64* osc, u64 kres = 1, int k_id = -1);
void add(const ckks_ctx* c, const u64* a, const u64* b, u64* o, int nlimbs, const int* ids, int lpp);
void sub(const ckks_ctx* c, const u64* a, const u64* b, u64* o, int nlimbs, const int* ids, int lpp);
void neg(const ckks_ctx* c, const u64* a, u64* o, int nlimbs, const int* ids, int lpp);
// bmod > 0: b broadcast, row k of a times row k % bmod of b (a plaintext times a batch)
void mul(const ckks_ctx* c, const u64* a, const u64* b, u64* o, int nlimbs, const int* ids, int lpp, int bmod = 0);
// o += a * b
void mul_acc(const ckks_ctx* c, const u64* a, const u64* b, u64* o, int nlimbs, const int* ids, int lpp);
// o = a * s[limb % lpp] (s residues, sp their Shoup companions; device arrays)
void mul_scalar(const ckks_ctx* c, const u64* a, const u64* s, const u64* sp, u64* o, int nlimbs, const int* ids,
                int lpp);
// by-value variants (no upload; usable inside stream capture)
// (a_pstride: row k of a at a + (k / lpp) * a_pstride + (k % lpp) * N; o contiguous)
void mul_scalar_v(const ckks_ctx* c, const u64* a, const ScalarVec& sv, u64* o, int nlimbs, const int* ids, int lpp,
                  size_t a_pstride = 0);
// out_k = a_k s1[r] - b_k s2[r] (r = k % lpp; s1 by value, s2/s2p device residues and Shoup
// companions; a rows as in mul_scalar_v, b and out contiguous)
void sub_mul2_scalar(const ckks_ctx* c, const u64* a, const u64* b, const ScalarVec& s1, const u64* s2,
                     const u64* s2p, u64* o, int nlimbs, const int* ids, int lpp, size_t a_pstride);
// (a_pstride: row k of a at a + (k / lpp) * a_pstride + (k % lpp) * N)
void add_scalar_v(const ckks_ctx* c, u64* a, const ScalarVec& sv, int nlimbs, const int* ids, int lpp,
                  size_t a_pstride = 0);
// a[limb][*] += v[limb]: adds the constant polynomial v in the NTT domain (device array v)
void add_const_term(const ckks_ctx* c, u64* a, const u64* v, int nlimbs, const int* ids);
// signed small ints (device int64 [N]) -> residues [nlimbs][N] (coefficient domain)
void small_to_rns(const ckks_ctx* c, const int64_t* v, u64* o, int nlimbs, const int* ids);
// o[i] = a[galois_src(i)] in the NTT domain
void automorph(const ckks_ctx* c, const u64* a, u64* o, int nlimbs, u64 g);
// o[limb] += s[limb % lpp] * automorph_g(a[limb]) (s = nullptr: o += automorph_g(a)), NTT domain
void automorph_acc(const ckks_ctx* c, const u64* a, u64* o, int nlimbs, u64 g, const u64* s, const u64* sp,
                   const int* ids, int lpp);
// X^{N/2} times a, NTT domain: pointwise by psi^((2 rev(i)+1) N/2)
void imult(const ckks_ctx* c, const u64* a, u64* o, int nlimbs, const int* ids, int lpp);
// centred lift of one coefficient-domain limb with prime `src_id` into nlimbs limbs
// (lpp > 0: row k lifts the source row k / lpp, at src + (k / lpp) * src_pstride, to prime ids[k % lpp])
void lift_centred(const ckks_ctx* c, const u64* src, int src_id, u64* o, int nlimbs, const int* ids, int lpp = 0,
                  size_t src_pstride = 0);
// out_i = (a_i - b_i) * s_i  (s device residues per limb index % lpp, Shoup companions sp); with
// a_pstride, row k of a is at a + (k / lpp) * a_pstride + (k % lpp) * N (b and out contiguous)
void sub_mul_scalar(const ckks_ctx* c, const u64* a, const u64* b, const u64* s, const u64* sp, u64* o,
                    int nlimbs, const int* ids, int lpp, size_t a_pstride = 0);
// fast base conversion, coefficient domain: in [nin][N] (limb stride in_stride words),
// out rows written at out + out_row[m]*N
// (prescaled: the inputs already carry the factor qhat_i^{-1}, see ConvTab::d_iscale)
void base_convert(const ckks_ctx* c, const ConvTab& t, const u64* in, size_t in_stride, u64* out,
                  size_t out_stride, int npoly, size_t in_poly_stride, size_t out_poly_stride,
                  bool prescaled = false);
// several conversions in one launch (e.g. every digit of a ModUp)
struct ConvJob {
    const u64* in;
    u64* out;
    const int *in_ids, *out_ids, *out_rows;
    const u64 *qinv, *qmod;
    const u64* inv_q;      // non-null: subtract v Q, v = round(sum_i xhat_i / q_i) (centred remainder)
    const u64* corr;
    int nin, nout, ngroups;
    size_t in_pstride, out_pstride;
    bool prescaled;        // inputs are x_i qhat_i^{-1} already (no product on load)
    const unsigned short* tcb;   // tensor-core form of the table (ConvTab::d_tcb, d_tcr)
    const u64* tcr;
    int tc_nin2, tc_S;
};
struct ConvJobs {
    static constexpr int MAX = 4;
    int n;
    ConvJob job[MAX];
};
void add_conv_job(ConvJobs& J, const ConvTab& t, const u64* in, u64* out, size_t in_pstride, size_t out_pstride,
                  bool prescaled = false);
void base_convert_jobs(const ckks_ctx* c, const ConvJobs& J, int npoly);
// tensor-core form of a conversion table (qmod [nout][nin], output moduli pm): the B image
// described at ConvTab::d_tcb, with its padded input count, group size and group count, and
// floor(2^88 / p_m) per output; empty when an output modulus is outside (2^39, 2^62)
std::vector<unsigned short> conv_tc_image(const std::vector<u64>& qmod, const std::vector<u64>& pm, int nin, int nout,
                                          int& nin2, int& S, int& groups, std::vector<u64>& r24p);
// the launch can run on the tensor cores (ctx->conv_tc, N >= 128, every job has its image)
bool conv_tc_eligible(const ckks_ctx* c, const ConvJobs& J);
void base_convert_tc_jobs(const ckks_ctx* c, const ConvJobs& J, int npoly);
// bounded device waits that ran out since the last call (the count is cleared); synchronous
unsigned take_device_faults();
unsigned peek_device_faults();   // the same count, not cleared
// test hook: withhold the tensor-core conversion's MMAs so that its bounded waits run out
void set_tc_withhold(bool on);
// key-switch inner product: D [ndig][next][N], key rows krow[e] of [ndig][nall][N];
// ob/oa [next][N] = sum_d D_d(sigma_g) * key_d ; g = 1 means no automorphism
// x0 (optional, rows [x0rows][N] with the primes of the first x0rows extended limbs): ob row e
// += s[e] * x0[e](sigma_g) for e < x0rows (s null: unscaled), the automorphed c0 term of a
// rotation, gathered with the same permutation as D; x1 (optional) likewise into oa (the
// P-lifted d0, d1 of a relinearisation, g = 1)
// (bt: a batch of bt.nb ciphertexts switched with the same key, D at + t dstr, ob / oa at + t ostr,
// x0 / x1 at + t xstr; at most 4 digits)
void ks_inner(const ckks_ctx* c, const u64* D, int ndig, int next, const int* ext_ids, const u64* kb,
              const u64* ka, u64* ob, u64* oa, u64 g, bool accumulate = false, const u64* x0 = nullptr,
              int x0rows = 0, const u64* s = nullptr, const u64* sp = nullptr, const u64* x1 = nullptr,
              const KsBatch& bt = KsBatch());
// d0 = a0 b0, d1 = a0 b1 + a1 b0 (d [2][nl][N]), d2 = a1 b1 (e [nl][N]) over nl limbs with
// primes ids[0..nl); a, b [2][nl][N]; for a batch of nb ciphertexts, ciphertext t's operands at
// a + t ab_bstride, b + t ab_bstride, d + t d_bstride, e + t e_bstride
void tensor(const ckks_ctx* c, const u64* a, const u64* b, u64* d, u64* e, int nl, const int* ids, int nb = 1,
            size_t ab_bstride = 0, size_t d_bstride = 0, size_t e_bstride = 0);
// o += a * s[limb % lpp] (s residues, sp their Shoup companions; device arrays); o_pstride: row k
// of o at o + (k / lpp) * o_pstride + (k % lpp) * N (a contiguous)
void mul_scalar_acc(const ckks_ctx* c, const u64* a, const u64* s, const u64* sp, u64* o, int nlimbs, const int* ids,
                    int lpp, size_t o_pstride = 0);
// uniform residues in the NTT domain drawn from the counter stream (see ckks.h)
void sample_uniform(const ckks_ctx* c, u64* o, int nlimbs, const int* ids, u64 key);
void sample_small(const ckks_ctx* c, int64_t* o, u64 key, int kind /*0 ternary, 1 gauss*/);
}  // namespace kern

// host helpers shared by the translation units
namespace hostmath {
u64 mulmod(u64 a, u64 b, u64 q);
u64 powmod(u64 a, u64 e, u64 q);
u64 invmod(u64 a, u64 q);
u64 shoup(u64 w, u64 q);
u64 from_signed(int64_t v, u64 q);
DevMod make_mod(u64 q);
bool is_prime(u64 n);
u64 splitmix_mix(u64 z);
u64 stream_key(u64 seed, u64 tag);
u64 stream_word(u64 key, u64 i);
long long llround_away(double x);
}  // namespace hostmath

// chain construction (chain.cpp)
void build_chain(const ckks_params& P, std::vector<u64>& q, std::vector<u64>& p, std::vector<double>& delta);
u64 smallest_root_2n(u64 q, int n);
void gauss_table(double sigma, u64* t39);

// FP64 encoding and plan construction (fp64.cpp)
namespace fp64 {
std::vector<double> encode_slots(const std::vector<cplx>& z, int n);       // -> N real coeffs
std::vector<cplx> decode_slots(const std::vector<double>& f, int n);       // -> N/2 slots
typedef std::map<int, std::vector<cplx>> Diag;                            // offset -> vector
Diag s_product(const std::vector<int>& strides, int m, bool inverse);
std::vector<std::vector<int>> split_groups(const std::vector<int>& stages, int levels);
void ap_of_group(const std::vector<int>& strides, int m, int* a0, int* step, int* count);
std::vector<std::vector<cplx>> fused_conv_diagonals(const double* W, int cin, int cout, int f, int w, int n);
std::vector<cplx> dwconv_kernel_slots(const double* K, int c, int f, int w, int n);
Diag decompose_diag(int w, int m);
Diag fc_stoc_diagonals(const double* M, int n_out, int n_in, int n);
std::vector<double> decompose_kernels(const double* W, int cout, int cin, int f, int C, int t, int* f_out);
std::vector<cplx> real_cins_slots(const double* m, int C, int two_l);
std::vector<double> cins_to_reals(const std::vector<cplx>& z, int C, int two_l);
std::vector<double> cheb_interp_cos(double K, int r, int deg);
std::vector<double> power_to_cheb(const std::vector<double>& c, double alpha, double beta);
int default_bsgs_B(int count);
int boot_bsgs_B(int count);
}  // namespace fp64

