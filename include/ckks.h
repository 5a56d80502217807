/*
 * ckks.h -- C ABI of the GB300 RNS-CKKS library for CinS conv2d fused with
 * bootstrapping (NeuJeans, arXiv 2312.04356).
 *
 * Scheme: RNS-CKKS (Sec. 2.1: KeyGen / Enc / Dec / Eval, HE ops "OpName(ct, x)",
 * HRot), bootstrapping ModRaise -> CtoS -> ModEval -> StoC (Sec. 2.4), CinS
 * encoding (Sec. 3), conv2d by diagonal BSGS (Sec. 2.5, Eq. 3, Eq. 7), fusion of
 * the conv with StoC2 (Sec. 4, Eq. 8) and the Alg. 1 block.
 *
 * Conventions
 *  - Ring Z_q[X]/(X^N + 1).  A polynomial at level l has l+1 RNS limbs mod
 *    q_0..q_l; the library stores them on the device limb-major, uint64
 *    [limb][N], in the NTT (evaluation) domain, bit-reversed order.  Arrays that
 *    cross this ABI through *_import_rns / *_export_rns are host arrays in the
 *    COEFFICIENT domain, same [limb][N] layout (a ciphertext is [2][l+1][N]:
 *    c0 then c1), residues in [0, q_i).
 *  - Slots: z_j = m(zeta^(5^j)), zeta = exp(pi i / N), j < N/2 (Sec. 2.2);
 *    HRot(ct, r) moves slot j + r to slot j (Galois element 5^r mod 2N).
 *  - Every ciphertext carries a level and a scale (double).  Each level has a
 *    canonical scale Delta_l with Delta_{l-1} = Delta_l^2 / q_l inside each of
 *    the two prime segments (bootstrapping levels, circuit levels).
 *  - Handles are opaque and owned by the caller, who creates and destroys them;
 *    no call takes ownership of its arguments.  Inputs are const; output
 *    handles are overwritten (their device storage is resized as needed).
 *    Output handles may alias inputs unless stated otherwise.
 *  - All device work is enqueued on the stream given to ckks_ctx_create (and, for
 *    independent work inside one call, on side streams that the call joins back to
 *    it before returning; see ckks_ctx_set_side_streams); calls return once the
 *    work is enqueued unless stated otherwise.  ckks_sync waits and reports
 *    deferred device errors.  A handle may only be used with the context that
 *    created it, and a context by one host thread at a time (the serving runtime's
 *    worker replays recorded graphs and does not touch the context's state).
 *  - Return value: CKKS_OK (0) or one of the CKKS_E* codes; no exceptions cross
 *    the ABI.  ckks_last_error(ctx) describes the last failure on that context.
 *  - Randomness: SplitMix64 used as a counter generator; stream key
 *    mix(seed ^ mix(tag + 0x9E3779B97F4A7C15)), word i = mix(key + (i+1)*gamma),
 *    with the tag layout kind<<56 | a<<16 | b.  Uniform residues are drawn
 *    directly in the NTT domain as (w[2k] << 64 | w[2k+1]) mod q, k = prime_id*N + j.
 */
#ifndef CKKS_GB300_H
#define CKKS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CKKS_OK 0
#define CKKS_EINVAL 1   /* bad argument, shape, level or scale mismatch */
#define CKKS_ENOKEY 2   /* a needed rotation / conjugation / relinearisation key is absent */
#define CKKS_ELEVEL 3   /* not enough levels left for the operation */
#define CKKS_ENOMEM 4   /* device allocation failed */
#define CKKS_ETIMEOUT 5 /* a bounded device wait gave up */
#define CKKS_ECUDA 6    /* any other CUDA error */

typedef struct ckks_ctx ckks_ctx;
typedef struct ckks_keys ckks_keys;
typedef struct ckks_ct ckks_ct;
typedef struct ckks_pt ckks_pt;
typedef struct ckks_ptset ckks_ptset;
typedef struct ckks_boot ckks_boot;

/* Parameter set (Table 3 and the RNS-CKKS chain).
 *   log_n       log2 N
 *   n_q         Q-limbs; levels 0..n_q-1
 *   dnum        key-switching digits; alpha = ceil(n_q / dnum) limbs per digit
 *   n_p         special primes (0 = alpha)
 *   q0_bits     base prime q_0 = largest prime < 2^q0_bits, = 1 mod 2N
 *   scale_bits  circuit levels 1..n_q-1-n_boot: Delta = 2^scale_bits
 *   p_bits      special primes: next largest primes < 2^p_bits, = 1 mod 2N
 *   boot_bits, n_boot  the top n_boot levels use base 2^boot_bits (0 = none)
 *   h           Hamming weight of the secret (0 = uniform ternary)
 *   sigma       Gaussian error deviation (truncated at |e| <= 19)
 * Scaling primes: within a segment of base 2^b, from its top level down, q_l is
 * the unused prime = 1 mod 2N nearest to Delta_l^2 / 2^b (ties: the smaller),
 * Delta_top = 2^b, Delta_{l-1} = Delta_l^2 / q_l.  The bootstrapping segment is
 * chosen first.  psi_i is the smallest primitive 2N-th root of unity mod q_i. */
typedef struct ckks_params {
    int log_n, n_q, dnum, n_p;
    int q0_bits, scale_bits, p_bits;
    int boot_bits, n_boot;
    int h;
    double sigma;
} ckks_params;

/* ---- context ------------------------------------------------------------ */
/* Builds primes, roots and twiddle tables on `cuda_stream` (a cudaStream_t, NULL =
 * legacy default stream).  seed drives every random draw of keys and encryption.
 * Errors: CKKS_EINVAL (log_n outside 3..17, n_q < 1, ...), CKKS_ENOMEM, CKKS_ECUDA. */
int ckks_ctx_create(const ckks_params* params, uint64_t seed, void* cuda_stream, ckks_ctx** out);
int ckks_ctx_destroy(ckks_ctx* ctx);
const char* ckks_last_error(const ckks_ctx* ctx);
/* Waits for the context's stream; returns CKKS_ECUDA on a deferred device error and
 * CKKS_ETIMEOUT while bounded device waits that ran out are on record for the device (see
 * ckks_ctx_take_device_faults). */
int ckks_sync(ckks_ctx* ctx);
/* Host copies of the chain: q[n_q], p[n_p], psi[n_q + n_p] (q's then p's), delta[n_q].
 * Any pointer may be NULL. */
int ckks_ctx_info(const ckks_ctx* ctx, uint64_t* q, uint64_t* p, uint64_t* psi, double* delta);
/* The 39-entry cumulative table of the Gaussian sampler (entry k: values <= k - 19). */
int ckks_ctx_gauss_table(const ckks_ctx* ctx, uint64_t* table39);

/* ---- device memory -------------------------------------------------------- */
/* A caller-provided device allocator: alloc(user, bytes, cuda_stream) returns device memory
 * (16-byte aligned; NULL = out of memory) for work enqueued on cuda_stream;
 * free(user, ptr, bytes, cuda_stream) gives it back when the library has enqueued its last
 * use on that stream, so the allocator may hand it out again for later work on the same
 * stream without waiting (the contract of a stream-ordered caching allocator such as
 * PyTorch's).  The callbacks run on the calling host thread and must not call this library. */
typedef void* (*ckks_alloc_fn)(void* user, size_t bytes, void* cuda_stream);
typedef void (*ckks_free_fn)(void* user, void* ptr, size_t bytes, void* cuda_stream);
/* Device memory of this context's later calls (ciphertexts, plaintexts, keys, temporaries)
 * comes from alloc / free_fn (both NULL: the library's default, stream-ordered cudaMallocAsync
 * on the device's default memory pool, whose release threshold it raises so the pool
 * caches).  With a caller allocator every call keeps all of its work on the context's stream
 * (no side streams, see ckks_ctx_set_side_streams).  Memory of work recorded into a CUDA
 * graph (ckks_*_graph_create, ckks_block_batch_create, the serving runtime) still comes from
 * the stream-ordered pool: it must live as long as the graph.  The constant tables built by
 * ckks_ctx_create come from cudaMalloc.  A buffer is freed through the allocator that
 * provided it, so the allocator may be changed at any time; `user` is passed back unchanged
 * and must stay valid while buffers from it are alive.
 * Errors: CKKS_EINVAL (only one of alloc / free_fn given). */
int ckks_ctx_set_allocator(ckks_ctx* ctx, ckks_alloc_fn alloc, ckks_free_fn free_fn, void* user);
/* Usage of the device's default memory pool (the library's default allocator): stats4 =
 * bytes in use now, the most in use since the last reset, bytes reserved now, the most
 * reserved since the last reset.  reset_high != 0 first resets both high-water marks to the
 * current values.  Synchronises the context's stream. */
int ckks_ctx_pool_stats(ckks_ctx* ctx, int reset_high, uint64_t* stats4);

/* ---- measurement (the paper's per-phase breakdown, Table 2) ---------------- */
/* Switch per-kernel CUDA-event timing on or off (off by default).  While on, every
 * kernel launch is bracketed by two events on the context's stream. */
int ckks_ctx_set_timing(ckks_ctx* ctx, int on);
/* counters[0..5] = kernel launches, key switches, PMults, HRots, HMults, rescales
 * since the context was created (or the last reset) */
int ckks_ctx_counters(const ckks_ctx* ctx, int64_t* counters6);
int ckks_ctx_reset_counters(ckks_ctx* ctx);
/* Per-kernel statistics gathered while timing was on, as a JSON object
 * {"kernel": [launches, total_ms, algorithmic_bytes], ...} (bytes: the minimum each
 * launch must read and write, summed) written to buf (NUL-terminated, truncated
 * to cap bytes); *len receives the full length.  Synchronises the stream. */
int ckks_ctx_kernel_stats(ckks_ctx* ctx, char* buf, int cap, int* len);

/* Autotuner: times each NTT launch variant (two passes of 8 stages with 16 values per thread,
 * 16 or 4 sub-problems per CTA and 3 or 4 resident CTAs per SM, or 4 values per thread; or
 * the whole transform in one launch by a cluster of 8 CTAs that exchange the half-transformed
 * data through distributed shared memory) for limb counts 1, 2, 7, 14, 24, 48, 96, 192
 * (forward + inverse, `reps` repetitions, 0 = 3) and keeps the fastest per size class for
 * this context.  All variants compute the same residues.  choice8 (may be NULL) receives the
 * chosen variant per class (0: 16 sub-problems / 80 registers, 1: 16 / 64, 2: 4 / 80,
 * 3: 4 / 64, 4: 4 values per thread, 5: one-launch cluster; -1: default).  Only N = 2^16 has
 * variants.  Synchronises the stream. */
int ckks_autotune(ckks_ctx* ctx, int reps, int32_t* choice8);
/* Use one NTT variant (0..5 as above) for every size, or -1 for the default rule. */
int ckks_ctx_set_ntt_variant(ckks_ctx* ctx, int variant);
/* Set the variant of each size class (choice8 as ckks_autotune returns it, -1..5 each), e.g.
 * to replay an earlier tuning without timing again. */
int ckks_ctx_set_ntt_choices(ckks_ctx* ctx, const int32_t* choice8);
/* Launch mode of the context's kernels.  on != 0 (the default): kernels launched outside a
 * CUDA graph capture use programmatic stream serialization, so the next kernel is set up
 * while the previous one drains; each kernel waits for its predecessors to complete before
 * its first memory access, so results are identical either way.  Captured launches are
 * always plain.  on == 0: plain launches everywhere. */
int ckks_ctx_set_pdl(ckks_ctx* ctx, int on);
/* Independent work inside one operation (the giant steps of an HMatmul, the Chebyshev
 * leaves, the products of one generation of the Chebyshev power ladder, the division nodes
 * of one height) runs on up to four side streams joined back by events (parallel branches of
 * a captured graph) when on != 0 (the default); on == 0 keeps everything on the context's
 * stream, e.g. so that per-kernel event timing measures each kernel alone.  Results are
 * identical either way. */
int ckks_ctx_set_side_streams(ckks_ctx* ctx, int on);
/* on != 0: the independent products of one generation of a Chebyshev evaluation's power
 * ladder (T_3 and T_4; T_5 .. T_8) that are taken at the same level run as one lockstep batch
 * (one launch per kernel for all of them, the relinearisation key read once) instead of side
 * by side on the side streams; results are identical either way.  Off by default. */
int ckks_ctx_set_inner_batching(ckks_ctx* ctx, int on);
/* mode 1 (the default) or 2: base conversions (ModUp, ModDown, ModDown fused with the
 * rescale; Sec. 2's hybrid key switching) run on the tensor cores: the 64-bit words and the
 * table are cut into 8-bit chunks, the chunk products are summed by FP16 x FP16 -> FP32 MMAs
 * (every sum an integer below 2^23, so exact) and reassembled and reduced mod p on the
 * integer pipe, by one (mode 1) or two (mode 2) threads per coefficient.  mode 0: 64-bit
 * multiply-adds on the integer pipe.  Results are identical in every mode.  Errors:
 * CKKS_EINVAL (mode outside 0..2). */
int ckks_ctx_set_tensor_conversion(ckks_ctx* ctx, int mode);
/* *count = the number of bounded waits inside the library's kernels (an mbarrier that a
 * tensor-core or bulk-copy completion should have signalled within ~1 s) that ran out on the
 * context's device since the last call, which clears it.  A kernel whose wait runs out
 * records it here, releases its tensor memory and returns; its outputs are then undefined.
 * Zero in normal operation.  Synchronises the context's stream. */
int ckks_ctx_take_device_faults(ckks_ctx* ctx, uint32_t* count);
/* Test hook for the bounded waits (no counterpart in the paper): on != 0 makes the
 * tensor-core base conversion on the context's device withhold its MMAs and their completion
 * signal, so that each of its CTAs gives up waiting after ~1 s, records the timeout, releases
 * its tensor memory and returns (outputs undefined); on == 0 restores normal operation.  The
 * device and the context stay usable.  Synchronises the context's stream.  For tests only. */
int ckks_debug_withhold_tensor_commit(ckks_ctx* ctx, int on);

/* ---- keys (Sec. 2.1 KeyGen) ----------------------------------------------- */
/* Secret key s (h-sparse or uniform ternary), public key (-a s + e, a) over Q_L,
 * relinearisation key, rotation keys for every step in rot_steps (mod N/2, 0 and
 * duplicates ignored) and, if want_conj, the conjugation key.  Switching keys are
 * hybrid: per digit d, (b_d, a_d) over Q_L u P with b_d = -a_d s + e_d + [P]_{q_i} s'
 * on the digit's limbs.  Keys stay resident on the device. */
int ckks_keygen(ckks_ctx* ctx, const int32_t* rot_steps, int n_rot, int want_conj, ckks_keys** out);
int ckks_keys_add_rotations(ckks_ctx* ctx, ckks_keys* keys, const int32_t* rot_steps, int n_rot);
int ckks_keys_destroy(ckks_keys* keys);
/* host copy of the secret key's coefficients (int64[N], values in {-1, 0, 1}) */
int ckks_keys_export_secret(ckks_ctx* ctx, const ckks_keys* keys, int64_t* s);

/* ---- handles ------------------------------------------------------------ */
int ckks_ct_create(ckks_ctx* ctx, ckks_ct** out);
int ckks_ct_destroy(ckks_ct* ct);
int ckks_ct_info(const ckks_ct* ct, int* level, double* scale);
int ckks_ct_set_scale(ckks_ct* ct, double scale);
/* host [2][level+1][N] coefficient domain <-> device (NTT domain inside) */
int ckks_ct_import_rns(ckks_ctx* ctx, const uint64_t* host, int level, double scale, ckks_ct* out);
int ckks_ct_export_rns(ckks_ctx* ctx, const ckks_ct* ct, uint64_t* host);
/* Copies src into dst's existing device buffer (same level required; dst keeps its
 * address).  Every other call that writes a ciphertext handle may give it a new buffer,
 * which matters to a CUDA graph that recorded the old one (see ckks_block_graph_create). */
int ckks_ct_copy_into(ckks_ctx* ctx, const ckks_ct* src, ckks_ct* dst);
int ckks_pt_create(ckks_ctx* ctx, ckks_pt** out);
int ckks_pt_destroy(ckks_pt* pt);
int ckks_pt_info(const ckks_pt* pt, int* level, double* scale);
/* host [level+1][N] coefficient domain: the bit-exact parity path for plaintexts */
int ckks_pt_import_rns(ckks_ctx* ctx, const uint64_t* host, int level, double scale, ckks_pt* out);
int ckks_pt_export_rns(ckks_ctx* ctx, const ckks_pt* pt, uint64_t* host);

/* ---- encoding (Sec. 2.2, Sec. 3.3.1) -------------------------------------- */
#define CKKS_SLOT 0       /* n <= N/2 complex slots (re, im); f = (1/N)(conj(U)^T z + U^T conj(z)) */
#define CKKS_COEFF 1      /* n <= N real coefficients (re) */
#define CKKS_CINS_REAL 2  /* real CinS (Eq. 5): n = C * slice_len reals, slice_len = 2l, C = N / 2l;
                             slot i*l + j = sum_k m_i[k] omega_{4l}^(5^j k) (Appendix A) */
/* FP64 on the host; coefficients round(scale * f) (halves away from zero), |.| < 2^62. */
int ckks_encode(ckks_ctx* ctx, const double* re, const double* im, int n, int level, double scale,
                int kind, int slice_len, ckks_pt* out);
/* Exact CRT to centred integers, divide by the plaintext's scale, then the inverse
 * of `kind`.  Blocks until the data is on the host. */
int ckks_decode(ckks_ctx* ctx, const ckks_pt* pt, int kind, int slice_len, double* re, double* im, int n);

/* Data organisation of Sec. 3.3.2: each of the c channels of img ([c][w0][w0] doubles)
 * is zero-padded to w x w (image top-left), flattened row-major and placed in slice i
 * (2l = w^2 reals, C = N / w^2 >= c slices), then real-CinS encoded (Eq. 5). */
int ckks_encode_image(ckks_ctx* ctx, const double* img, int c, int w0, int w, int level, double scale,
                      ckks_pt* out);
/* Inverse reading into out[c][w0][w0].  from_coeff = 0: real-CinS slots.  from_coeff = 1:
 * the coefficient-encoded output of the fused conv, channel i at coefficients
 * k*C + rev_C(i), k < w^2 (Thm. 2 with Y = X^C).  Blocks until the data is on the host. */
int ckks_decode_image(ckks_ctx* ctx, const ckks_pt* pt, int from_coeff, int c, int w0, int w, double* out);

/* ---- encryption (Sec. 2.1 Enc / Dec) -------------------------------------- */
/* pk: (u b + e0 + m, u a + e1), u uniform ternary, e0, e1 Gaussian; streams tagged by nonce */
int ckks_encrypt(ckks_ctx* ctx, const ckks_keys* keys, const ckks_pt* pt, uint64_t nonce, ckks_ct* out);
/* sk: (-a s + e + m, a), a uniform over the level's limbs */
int ckks_encrypt_sk(ckks_ctx* ctx, const ckks_keys* keys, const ckks_pt* pt, uint64_t nonce, ckks_ct* out);
/* m = c0 + c1 s */
int ckks_decrypt(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* ct, ckks_pt* out);

/* ---- HE ops (Sec. 2.1 "OpName(ct, x)") ------------------------------------ */
/* HAdd / HSub: same level, scales equal to 2^-30 relative */
int ckks_add(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, ckks_ct* out);
int ckks_sub(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, ckks_ct* out);
/* PMult without rescale: scale = ct.scale * pt.scale; pt must be at the ct's level */
int ckks_mul_plain(ckks_ctx* ctx, const ckks_ct* ct, const ckks_pt* pt, ckks_ct* out);
/* HMult: tensor, relinearise (key switch of c1 c1'), no rescale; same level */
int ckks_mul_relin(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* a, const ckks_ct* b, ckks_ct* out);
/* CMult by an integer (scale unchanged) */
int ckks_mul_int(ckks_ctx* ctx, const ckks_ct* ct, int64_t c, ckks_ct* out);
/* CAdd: every slot += c, as llround(c * scale) added to the constant coefficient */
int ckks_add_const(ckks_ctx* ctx, const ckks_ct* ct, double c, ckks_ct* out);
/* every slot times i (polynomial times X^(N/2)) */
int ckks_imult(ckks_ctx* ctx, const ckks_ct* ct, ckks_ct* out);
/* Rescale (Sec. 2.4): c'_i = (c_i - [c_l]_{q_l, centred}) q_l^{-1}; scale / q_l */
int ckks_rescale(ckks_ctx* ctx, const ckks_ct* ct, ckks_ct* out);
/* drop limbs above `level` (scale unchanged) */
int ckks_mod_drop(ckks_ctx* ctx, const ckks_ct* ct, int level, ckks_ct* out);
/* per level: times llround((Delta_{l-1} * q_l) / scale), rescale, scale := Delta_{l-1} */
int ckks_level_down(ckks_ctx* ctx, const ckks_ct* ct, int level, ckks_ct* out);
/* ModRaise (Sec. 2.4): level-0 ct, centred residues mod q_0 lifted to every limb; scale kept */
int ckks_mod_raise(ckks_ctx* ctx, const ckks_ct* ct, ckks_ct* out);
/* HRot for each step (Sec. 2.1): one ModUp of c1 shared by all steps ("hoisted");
 * per step: Galois automorphism of the raised digits, inner product with the key,
 * ModDown.  outs[i] receives step i; outs must not alias `in`.  CKKS_ENOKEY if a key
 * is missing. */
int ckks_rotate_hoisted(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const int32_t* steps,
                        int n, ckks_ct* const* outs);
/* conjugation (Galois element 2N - 1) */
int ckks_conjugate(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* ct, ckks_ct* out);

/* ---- BSGS linear maps (Sec. 2.5, Eq. 3) ----------------------------------- */
/* A map on the N/2 slots with diagonals at offsets a0 + step*i (mod N/2), i < count,
 * evaluated as sum_g rot_{a0+step*g*B}( sum_b pt_{g,b} (.) rot_{step*b}(ct) ) with
 * pt_{g,b} = diag_{a0+step(gB+b)} pre-rotated right by a0 + step*g*B.  Absent
 * (g, b) entries are zero diagonals.  All plaintexts sit at `level`. */
int ckks_ptset_create(ckks_ctx* ctx, int a0, int step, int count, int bsgs_B, int level, double scale,
                      ckks_ptset** out);
int ckks_ptset_destroy(ckks_ptset* ps);
/* host [level+1+np][N] coefficient-domain limbs of pt_{g,b} over Q_level then the special
 * primes (copied): BSGS diagonals are kept over Q_level u P for double hoisting */
int ckks_ptset_set_rns(ckks_ctx* ctx, ckks_ptset* ps, int g, int b, const uint64_t* host);
int ckks_ptset_info(const ckks_ptset* ps, int* a0, int* step, int* count, int* bsgs_B, int* level,
                    double* scale, int* n_pts);
/* distinct non-zero rotation steps the map needs (baby then giant); *n_out = count */
int ckks_ptset_rotations(const ckks_ptset* ps, int32_t* steps, int cap, int* n_out);
/* evaluate the map, no rescale */
int ckks_bsgs(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* ct, const ckks_ptset* ps, ckks_ct* out);

/* Fused CinS conv2d (Sec. 4.2): plaintexts of the diagonals of K' = S' K^, where K^ is
 * the C x C slice matrix of DFT'_{2l}(k_{o,i}) (kernel vectors of Fig. 1 with 'same'
 * padding, cross-correlation) and S' the slice matrix of StoC2 = S_{N/2 <- l}.
 * weights: [cout][cin][f][f] doubles; channel i of the input sits in slice i of a
 * w x w padded image (w a power of two, 2l = w^2, C = N / w^2 >= cin, cout).
 * BSGS over offsets d*l, d < C; bsgs_B = 0 picks 2^ceil(log2(C)/2). */
int ckks_ptset_conv_fused(ckks_ctx* ctx, const double* weights, int cin, int cout, int f, int w, int level,
                          double pt_scale, int bsgs_B, ckks_ptset** out);
/* Alg. 1, conv step: BSGS with the fused diagonals, then rescale.  The output is
 * coefficient-encoded: coefficient k*C + rev_C(i) holds Delta * o_i[k] (Thm. 2, Y = X^C). */
int ckks_conv2d_cins(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const ckks_ptset* conv,
                     ckks_ct* out);

/* Decomposed downsampling conv2d (Alg. 2's decomposed conv).  W[cout][cin][f][f] is a stride-2
 * cross-correlation with zero padding f/2 (PyTorch semantics, even image width).  Input
 * ciphertext t holds channels tC .. tC + C - 1 (C = N / w_in^2) as the stride-2 tail of
 * ckks_boot_create leaves them: 4C polyphase slices of width w_in/2.  The set rewrites the
 * taps of those channels as a unit-stride conv over the polyphase slices (tap (a, b) ->
 * slice 4i + q + 2p, offset (dy, dx) with a - f/2 = 2 dy + p, b - f/2 = 2 dx + q) and fuses
 * it with StoC2 at width w_in/2 like ckks_ptset_conv_fused (cout <= 4C outputs).  Summing
 * the sets' BSGS over t = 0, 1, ... gives the stride-2 conv (ckks_block_multi). */
int ckks_ptset_conv_fused_s2(ckks_ctx* ctx, const double* weights, int cin, int cout, int f, int w_in, int t,
                             int level, double pt_scale, int bsgs_B, ckks_ptset** out);
/* Downsampling depthwise conv2d (Sec. 3.3.4): K[c][f][f] (host, row-major, read during the
 * call) are the stride-2 kernels of channels 0 .. c - 1, output channel o = input channel o;
 * the set is ckks_ptset_conv_fused_s2 with the diagonal weights W[o][o] = K[o] (cin = cout =
 * c <= 4C: the channels of up to four input ciphertexts, which fill one output ciphertext;
 * larger layers split their channels into such groups).  Average pooling with stride 2 is
 * the case of equal kernels 1 / f^2 (zero padding f/2 counted in the mean).  CKKS_EINVAL for
 * c < 1, f < 1, c^2 f^2 > 2^28, and whatever ckks_ptset_conv_fused_s2 refuses. */
int ckks_ptset_dwconv_fused_s2(ckks_ctx* ctx, const double* K, int c, int f, int w_in, int t, int level,
                               double pt_scale, int bsgs_B, ckks_ptset** out);
/* The Alg. 2 decomposition as one plaintext set: diagonals at offsets b w/4,
 * |b| < w (0/1 masks), encoded at (level, scale); the slot permutation described at
 * ckks_boot_create.  Apply with ckks_bsgs + ckks_rescale. */
int ckks_ptset_decompose(ckks_ctx* ctx, int w, int level, double scale, int bsgs_B, ckks_ptset** out);

/* Fully-connected layer fused with the whole StoC (Sec. 4.3: slot encoding is CinS with
 * l = 1, so the FC matrix merges with all of S_{N/2<-1}).  The input holds x (n_in reals,
 * n_in a power of two) in slots 0 .. n_in - 1 and zeros elsewhere; the output holds
 * y = M x (M row-major [n_out][n_in], n_out <= N/2) in its coefficients 0 .. n_out - 1
 * (coefficient encoding: ready for ModRaise, or for ckks_decode with CKKS_COEFF).  The
 * set holds the n_in diagonals of V M on x replicated with period n_in (d_o[i] =
 * (V M)[i][(i + o) mod n_in]); ckks_fc_stoc replicates x with log2(N / 2n_in) rotations
 * by -n_in 2^t, then BSGS + rescale (one level).  Rotation keys: those of the set and the
 * replication steps. */
int ckks_ptset_fc_stoc(ckks_ctx* ctx, const double* M, int n_out, int n_in, int level, double pt_scale, int bsgs_B,
                       ckks_ptset** out);
int ckks_fc_stoc(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const ckks_ptset* fc, int n_in,
                 ckks_ct* out);

/* Depthwise conv2d (Sec. 3.3.4; Table 1: 1 PMult, 0 HRot, 1 level): the c kernels
 * K[c][f][f] (cross-correlation, 'same' padding, kernel vectors of Fig. 1) packed in one
 * real-CinS plaintext <k_1 | ... | k_C>, so that one PMult gives k_i * i_i in every slice
 * (Eq. 6).  ckks_dwconv_cins = PMult + rescale; the output stays real-CinS.  Average
 * pooling with stride 1 is the case of equal kernels 1 / f^2; with stride 2 it is
 * ckks_ptset_dwconv_fused_s2 (a downsampling conv). */
int ckks_encode_dwconv_kernel(ckks_ctx* ctx, const double* K, int c, int f, int w, int level, double scale,
                              ckks_pt* out);
int ckks_dwconv_cins(ckks_ctx* ctx, const ckks_ct* in, const ckks_pt* kernel, ckks_ct* out);

/* ---- bootstrapping and the Alg. 1 block ----------------------------------- */
typedef struct ckks_boot_params {
    int w, w0, cout;      /* padded width, image width, output channels (masks) */
    int K;                /* |ModRaise overflow| < K */
    int r;                /* double-angle steps */
    int deg;              /* Chebyshev degree of the cosine */
    int ctos_levels, stoc_levels;
    double delta0;        /* scale of the level-0 ciphertext entering ModRaise */
    int stride;           /* 0 or 1; 2 when the next conv downsamples (Alg. 2, see below) */
} ckks_boot_params;
/* Builds: ModRaise scale q0*K_eff and drop constant c_drop = llround((Delta_{ld-1} q_ld) /
 * (q0 K)) with ld = L - ctos_levels, K_eff = (Delta_{ld-1} q_ld) / (q0 c_drop); CtoS =
 * T_{N/2}^{-1} in ctos_levels BSGS levels (largest stride first, plaintext scale q_l,
 * last level times 1/2); Chebyshev coefficients of cos(2 pi (K_eff y - 1/4) / 2^r);
 * padding masks times q0 / (2 pi delta0); StoC1 = S_{l <- 1} in stoc_levels levels.
 * stride = 2 (Alg. 2's decomposition and S_{l/4<-1}): after Re + i Im the tail applies
 * the decomposition (one HMatmul by the slot permutation sum_j (>> j l/4) calG_l (<< r_j),
 * r = (0, l/2, w/4, l/2 + w/4), calG_l of Appendix B, plaintexts at canonical scale; see
 * ckks_ptset_decompose) and StoC1 becomes S_{l/4 <- 1}: the output holds, in slice
 * 4i + q + 2p, the polyphase image x_i[p::2][q::2] of channel i as real CinS of width w/2.
 * Needs w >= 4 and an even w0; l_out is one level lower than with stride 1. */
int ckks_boot_create(ckks_ctx* ctx, const ckks_boot_params* bp, ckks_boot** out);
int ckks_boot_destroy(ckks_boot* bt);
/* info[0..7] = K_eff, s_raise, c_drop, l_drop, l_em, l_out, s_em, s_mask */
int ckks_boot_info(const ckks_boot* bt, double* info8);
int ckks_boot_rotations(const ckks_boot* bt, int32_t* steps, int cap, int* n_out);
/* ---- BSGS split per level (Sec. 2.6: an HMatmul with `count` diagonals as B baby steps
 * and ceil(count / B) giant steps).  Levels in evaluation order: the CtoS levels, the
 * stride-2 decomposition (if any), the StoC1 levels; n_out receives their number.
 * ckks_boot_create picks B by the cost model (B - 1) + 5 (G - 1) (HRots, a giant step
 * costing about five baby rotations under double hoisting).  The rotation keys a block
 * needs (ckks_boot_rotations) follow the splits in force. */
int ckks_boot_bsgs_splits(const ckks_boot* bt, int32_t* B, int cap, int* n_out);
/* Rebuild every level's plan with the given baby-step counts, 1 <= B[i] <= 32 (B above the
 * level's diagonal count means one giant step); n must equal the number of levels.
 * CKKS_EINVAL otherwise (plans unchanged). */
int ckks_boot_set_bsgs_splits(ckks_ctx* ctx, ckks_boot* bt, const int32_t* B, int n);
/* Autotuner: per level, times one HMatmul with rescale for B in {2, 4, ..., 32} (up to the
 * level's diagonal count) and the cost-model choice, `reps` runs each after one warm-up,
 * on a fresh encryption at the level's input level, with temporary switching keys for the
 * candidates' rotations (freed before the next level: at N = 2^16 a few GB at a time), and
 * keeps the fastest plan.  B_out (may be NULL, cap entries) receives the chosen counts.
 * Run it before generating the keys a block will use.  Op and launch counters are left
 * unchanged; synchronises the stream. */
int ckks_boot_tune_bsgs(ckks_ctx* ctx, ckks_boot* bt, int reps, int32_t* B_out, int cap, int* n_out);
/* replace one CtoS / StoC1 level, the EvalMod coefficients, or the masks
 * (used to feed identical plaintexts to two implementations) */
int ckks_boot_set_ctos(ckks_ctx* ctx, ckks_boot* bt, int i, const ckks_ptset* ps);
int ckks_boot_set_stoc(ckks_ctx* ctx, ckks_boot* bt, int i, const ckks_ptset* ps);
int ckks_boot_set_decomp(ckks_ctx* ctx, ckks_boot* bt, const ckks_ptset* ps);
int ckks_boot_set_coeffs(ckks_ctx* ctx, ckks_boot* bt, const double* coeffs, int deg);
int ckks_boot_set_masks(ckks_ctx* ctx, ckks_boot* bt, const ckks_pt* re, const ckks_pt* im);
/* ModRaise -> CtoS -> conjugate split (Re = ct + conj, Im = i (conj - ct)) -> scale drop
 * -> EvalMod(Re), EvalMod(Im) (Alg. 1, bootstrapping step). */
int ckks_bootstrap(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* bt, const ckks_ct* ct0,
                   ckks_ct* out_re, ckks_ct* out_im);
/* mask PMults, Re + i Im, HMatmul(S_{l<-1}) (Alg. 1, activation and StoC1 steps, without
 * HActivation) */
int ckks_stoc1(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* re, const ckks_ct* im, const ckks_boot* bt,
               ckks_ct* out);
/* one conv2d + bootstrap block: conv2d_cins -> bootstrap -> stoc1 */
int ckks_block(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const ckks_ptset* conv,
               const ckks_boot* bt, ckks_ct* out);
/* The same block over n_in input ciphertexts: sum_t BSGS(in[t], conv[t]) (HAdd, one
 * rescale) -> bootstrap -> stoc1.  With the plaintext sets of ckks_ptset_conv_fused_s2 this
 * is Alg. 2 from the decomposed convs to the end (the downsampling conv bootstraps one
 * ciphertext where a stride-1 conv followed by densify bootstraps s^2 = 4); with ckks_ptset_conv_fused sets over
 * different input channels it is the C_in > C block matrix-vector product (Sec. 3.3.3).
 * All inputs share level and scale, all sets share level and scale; 1 <= n_in <= 64. */
int ckks_block_multi(ckks_ctx* ctx, const ckks_keys* keys, int n_in, const ckks_ct* const* in,
                     const ckks_ptset* const* conv, const ckks_boot* bt, ckks_ct* out);

/* ---- CUDA graphs ------------------------------------------------------------- */
typedef struct ckks_graph ckks_graph;
/* Records one ckks_block (in -> out) into a CUDA graph.  Runs the block once eagerly
 * first (this sizes `out`), then captures a second run on the context's stream, whose
 * result is copied into out's device buffer; intermediates are allocated and freed inside
 * the graph.  The context must have been created on a non-default stream.  Each launch
 * recomputes the block from whatever `in` holds then; `in` and `out` must stay alive and
 * keep their device buffers while the graph exists: write new inputs with
 * ckks_ct_copy_into, not with calls that reassign the handle.  Launches of one graph run one at a time;
 * independent graphs (capture one per input) may run concurrently on different streams. */
int ckks_block_graph_create(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const ckks_ptset* conv,
                            const ckks_boot* bt, ckks_ct* out, ckks_graph** graph);
/* cudaGraphLaunch on `stream` (a cudaStream_t; NULL = the context's stream) */
int ckks_graph_launch(ckks_graph* graph, void* stream);
/* number of kernel launches one replay performs */
int ckks_graph_info(const ckks_graph* graph, int64_t* kernel_launches);
int ckks_graph_destroy(ckks_graph* graph);

/* ---- batched blocks ------------------------------------------------------------ */
/* B independent ciphertexts through the same block (conv set, bootstrap configuration):
 * one ckks_block graph per input (in[i] -> out[i], recorded as ckks_block_graph_create
 * does, so each input runs once eagerly first), spread round-robin over min(n_streams, B)
 * CUDA streams the batch owns, so that the small launches of different ciphertexts overlap.
 * The inputs and outputs must stay alive while the batch exists; each launch re-reads in[]
 * and overwrites out[].  CKKS_EINVAL for B outside 1..1024, n_streams outside 1..32, an
 * output that aliases an input or another output; otherwise what ckks_block_graph_create
 * returns. */
typedef struct ckks_batch ckks_batch;
int ckks_block_batch_create(ckks_ctx* ctx, const ckks_keys* keys, int B, const ckks_ct* const* in,
                            const ckks_ptset* conv, const ckks_boot* bt, ckks_ct* const* out, int n_streams,
                            ckks_batch** batch);
/* Launches the B graphs after the work already enqueued on the context's stream; the
 * context's stream then waits for all of them (so ckks_sync covers the batch).  Asynchronous. */
int ckks_batch_launch(ckks_batch* batch);
/* Waits for the context's stream, then frees the graphs, streams and events. */
int ckks_batch_destroy(ckks_batch* batch);

/* Lockstep batch (the paper's amortisation of the BSGS plaintexts, Sec. 2.5, and of the
 * key-switching keys, Sec. 2.1, over many ciphertexts): B ciphertexts of one shape (same level
 * and scale) through the same block (Alg. 1 without HActivation, as ckks_block computes it)
 * as ONE batch: every kernel of the block is launched once for all B ciphertexts, so each
 * switching key and plaintext diagonal streams from HBM about once per batch (the CTAs of the
 * B ciphertexts that read the same key words run side by side and share them through L2),
 * and every NTT, base conversion and elementwise launch covers B times the limbs.  Each out[i]
 * receives exactly the ciphertext ckks_block would give for in[i] (same residues).  Device
 * memory: about B times that of one block.  CKKS_EINVAL for B outside 1..1024, inputs of
 * different levels or scales, an output that aliases an input or another output. */
int ckks_block_batched(ckks_ctx* ctx, const ckks_keys* keys, int B, const ckks_ct* const* in,
                       const ckks_ptset* conv, const ckks_boot* bt, ckks_ct* const* out);
/* The same lockstep batch recorded as one CUDA graph (gather of in[], batched block, scatter
 * into out[]), after one eager run that sizes out[]; the rules of ckks_block_graph_create
 * apply to every in[i] and out[i]. */
int ckks_block_batched_graph_create(ckks_ctx* ctx, const ckks_keys* keys, int B, const ckks_ct* const* in,
                                    const ckks_ptset* conv, const ckks_boot* bt, ckks_ct* const* out,
                                    ckks_graph** graph);
/* The Alg. 2 layer of ckks_downsample_layer for B independent inputs as one lockstep batch:
 * input b is the n_in pairs re[b * n_in + t], im[b * n_in + t] (t < n_in; every pair at the
 * level and scale of an EvalMod output), all inputs share bt_in, conv[n_in] and bt_out; out[b]
 * receives exactly what ckks_downsample_layer gives for input b.  Errors as
 * ckks_downsample_layer and ckks_block_batched. */
int ckks_downsample_layer_batched(ckks_ctx* ctx, const ckks_keys* keys, int B, int n_in, const ckks_ct* const* re,
                                  const ckks_ct* const* im, const ckks_boot* bt_in, const ckks_ptset* const* conv,
                                  const ckks_boot* bt_out, ckks_ct* const* out);
/* Lockstep batches of ckks_bootstrap (out_re[b], out_im[b] from in[b]), ckks_eval_poly and
 * ckks_eval_relu (out[b] from in[b]): every input at the same level and scale, each output
 * exactly what the single-ciphertext call gives; errors as those calls and ckks_block_batched. */
int ckks_bootstrap_batched(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* bt, int B, const ckks_ct* const* in,
                           ckks_ct* const* out_re, ckks_ct* const* out_im);
int ckks_eval_poly_batched(ckks_ctx* ctx, const ckks_keys* keys, int B, const ckks_ct* const* in,
                           const double* coeffs, int deg, int basis, double a, double b, ckks_ct* const* out);
int ckks_eval_relu_batched(ckks_ctx* ctx, const ckks_keys* keys, int B, const ckks_ct* const* in,
                           const double* coeffs, const int* degs, int n_stages, ckks_ct* const* out);

/* ---- serving loop ----------------------------------------------------------------
 * Continuous batching of inference requests (no counterpart in the paper, whose
 * measurements are one image at a time; a server needs batched throughput).
 * A model is a chain of Alg. 1 blocks: block b runs ckks_block with convs[b], boots[b]
 * after a level drop of its input to convs[b]'s level.  For each of `slots` slots (a CUDA
 * stream, device and pinned staging buffers) and each model, ckks_server_add_model runs
 * one request eagerly (checking keys and levels and measuring the peak bytes of its
 * temporaries in the device memory pool: the model's footprint), then records the whole
 * request -- NTT of the input limbs, the blocks, iNTT of the output -- as a CUDA graph.
 * After ckks_server_start a worker thread admits queued requests in submission order
 * into free slots while the footprints of the requests in flight sum to at most
 * hbm_budget bytes (0: no limit), and retires each as its slot's stream completes.
 * The context (created on a non-default stream), keys, plaintext sets and bootstrapping
 * configurations must outlive the server and must not be modified while it runs; the
 * worker only launches the recorded graphs and copies, so other work may share the device.
 * Requests carry coefficient-domain limbs [2][level+1][N] (the ckks_ct_export_rns /
 * ckks_ct_import_rns format) at the model's input level and canonical scale; results
 * are returned in the same format at the last block's l_out.  Errors: CKKS_EINVAL (bad
 * model, level or scale, unknown request), CKKS_ENOKEY (a block needs a key `keys` lacks,
 * found by the eager run), CKKS_ENOMEM (a request of the model exceeds hbm_budget). */
typedef struct ckks_server ckks_server;
typedef struct ckks_server_params {
    int slots;               /* requests in flight at once, 1..64 */
    long long hbm_budget;    /* bytes of temporaries the requests in flight may hold; 0 = no limit */
} ckks_server_params;
#define CKKS_REQ_QUEUED 0
#define CKKS_REQ_RUNNING 1
#define CKKS_REQ_DONE 2
#define CKKS_REQ_FAILED 3
#define CKKS_REQ_CANCELLED 4
int ckks_server_create(ckks_ctx* ctx, const ckks_keys* keys, const ckks_server_params* sp, ckks_server** out);
int ckks_server_add_model(ckks_server* s, int n_blocks, const ckks_ptset* const* convs, const ckks_boot* const* boots,
                          int* model_id);
/* A model as a chain of layers over several ciphertexts (a ResNet-shaped network of Alg. 1
 * blocks and Alg. 2 downsampling layers).  Layer k maps its n_in ciphertexts (the previous
 * layer's n_out) to n_out ciphertexts; output j reads k of them, in_index[j k .. j k + k - 1]
 * (in_index NULL: all n_in in order, k = n_in), with the sets convs[j k .. j k + k - 1]:
 *   CKKS_LAYER_BLOCK: output j is the Alg. 1 block over its inputs with configuration boot
 *     (ckks_block for one input, the Sec. 3.3.3 block matrix-vector product of
 *     ckks_block_multi for several), each input first brought down to the sets' level;
 *   CKKS_LAYER_DOWNSAMPLE: output j is ckks_downsample_layer(bt_in = boot_in, bt_out = boot)
 *     over the EvalMod outputs of its inputs: the previous layer must be a block layer, and
 *     it then stops after its bootstrap (Alg. 2 consumes the Re / Im halves; no StoC1).
 * Requests carry [n_in][2][level + 1][N] limbs of the first layer's inputs and return
 * [n_out][2][l_out + 1][N] of the last layer's outputs (ckks_server_model_shape).  Recording,
 * footprint and errors as ckks_server_add_model, plus CKKS_EINVAL for a layer whose input
 * count differs from the previous layer's output count, an input index out of range, a
 * downsampling layer first or after another downsampling layer, or a missing configuration. */
#define CKKS_LAYER_BLOCK 0
#define CKKS_LAYER_DOWNSAMPLE 1
typedef struct ckks_server_layer {
    int kind;                          /* CKKS_LAYER_BLOCK or CKKS_LAYER_DOWNSAMPLE */
    int n_in, n_out;                   /* ciphertexts into and out of the layer, 1..64 */
    int k;                             /* inputs per output, 1..n_in (n_in when in_index is NULL) */
    const int* in_index;               /* [n_out][k] input indices, or NULL: every output reads all */
    const ckks_ptset* const* convs;    /* n_out * k conv sets, output-major */
    const ckks_boot* boot;             /* block: its configuration; downsampling: bt_out */
    const ckks_boot* boot_in;          /* downsampling: bt_in; block: ignored */
} ckks_server_layer;
int ckks_server_add_model_layers(ckks_server* s, int n_layers, const ckks_server_layer* layers, int* model_id);
/* shape2[0..1] = ciphertexts into and out of a request of the model */
int ckks_server_model_shape(const ckks_server* s, int model_id, int* shape2);
/* info[0..5] = input level, input scale, output level, output scale, footprint bytes, kernels per request */
int ckks_server_model_info(const ckks_server* s, int model_id, double* info6);
int ckks_server_start(ckks_server* s);
/* copies host_in; *request_id identifies the request from then on */
int ckks_server_submit(ckks_server* s, int model_id, const uint64_t* host_in, int level, double scale,
                       uint64_t* request_id);
int ckks_server_poll(ckks_server* s, uint64_t request_id, int* state);
/* waits until the request is DONE, FAILED or CANCELLED; CKKS_ETIMEOUT after timeout_s seconds */
int ckks_server_wait(ckks_server* s, uint64_t request_id, double timeout_s, int* state);
/* host_out NULL: only level and scale.  Otherwise copies the result and forgets the request. */
int ckks_server_result(ckks_server* s, uint64_t request_id, uint64_t* host_out, int* level, double* scale);
/* a queued request is dropped; a running one finishes on the device and its result is discarded */
int ckks_server_cancel(ckks_server* s, uint64_t request_id);
/* stats[0..7] = completed, failed, cancelled, p50 latency ms, p99 latency ms, mean latency ms,
 * most requests in flight at once, kernel launches (submission to completion, host clock) */
int ckks_server_stats(ckks_server* s, double* stats8);
int ckks_server_reset_stats(ckks_server* s);
const char* ckks_server_last_error(const ckks_server* s);
/* stops admitting, waits for the requests in flight, abandons the queued ones */
int ckks_server_destroy(ckks_server* s);

/* ---- the downsampling layer (Alg. 2) ------------------------------------------ */
/* Alg. 2 without HActivation, from the EvalMod outputs of the previous block: for each of
 * the n_in input ciphertexts, ckks_stoc1 with the stride-2 configuration bt_in (masks,
 * Re + i Im, decomposition, S_{l/4<-1}) and a level drop to the conv sets' level; then
 * ckks_block_multi over the decomposed conv sets (ckks_ptset_conv_fused_s2, t = 0 .. n_in-1)
 * with bt_out.  re[t], im[t] sit at bt_in's l_em with its s_em; 1 <= n_in <= 64. */
int ckks_downsample_layer(ckks_ctx* ctx, const ckks_keys* keys, int n_in, const ckks_ct* const* re,
                          const ckks_ct* const* im, const ckks_boot* bt_in, const ckks_ptset* const* conv,
                          const ckks_boot* bt_out, ckks_ct* out);
/* The same layer recorded as a CUDA graph, under the rules of ckks_block_graph_create
 * (non-default stream; inputs and out keep their buffers while the graph lives). */
int ckks_downsample_layer_graph_create(ckks_ctx* ctx, const ckks_keys* keys, int n_in, const ckks_ct* const* re,
                                       const ckks_ct* const* im, const ckks_boot* bt_in,
                                       const ckks_ptset* const* conv, const ckks_boot* bt_out, ckks_ct* out,
                                       ckks_graph** graph);

/* ---- polynomial evaluation (HActivation) --------------------------------- */
#define CKKS_BASIS_CHEB 0
#define CKKS_BASIS_POWER 1
/* p(x) for slots x in [a, b] (HActivation, Sec. 2.4.2).  CKKS_BASIS_CHEB: p = sum_k c_k T_k(y),
 * y = (2x - a - b) / (b - a); CKKS_BASIS_POWER: p = sum_k c_k x^k, re-expressed on the host in
 * FP64 as a Chebyshev series in y (well conditioned for moderate degrees only).  For [a, b] !=
 * [-1, 1] the variable y costs one level: x times llround(alpha Delta_(l-1) q_l / scale), alpha =
 * 2 / (b - a), rescaled onto the canonical scale, then -(a + b) / (b - a) added.  T_k from
 * T_{ceil(k/2)} T_{floor(k/2)} (baby and giant steps, Chebyshev division), each piece brought to
 * the canonical scale of its target level after one rescale; levels used: ceil(log2 deg) + 1
 * (+ 1 for the change of variable, + 1 when the evaluation crosses from the bootstrapping
 * segment of the chain into the circuit segment).  Errors: CKKS_EINVAL (deg < 1, a >= b, unknown basis),
 * CKKS_ELEVEL. */
int ckks_eval_poly(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const double* coeffs, int deg,
                   int basis, double a, double b, ckks_ct* out);

/* ---- rescale without device allocation ------------------------------------ */
/* The paper has no counterpart to this call; it exists for callers that cannot allocate
 * device memory while they run (graphs recorded without memory-pool nodes, serving loops
 * that forbid cudaMalloc because it may synchronise the device, hosts that give the
 * library a fixed memory budget).  It computes exactly what ckks_rescale computes, on
 * raw device arrays: d_in is a ciphertext at `level` ([2][level+1][N] uint64, NTT domain,
 * c0 then c1), d_out receives the rescaled ciphertext ([2][level][N], NTT domain); d_out
 * must not overlap d_in.  The caller tracks the scale (divide it by q_level).
 * Scratch comes from one static device array of 2^22 words (32 MiB) that every GPU loading
 * the library holds until exit; calls needing more than (2 level + 2) N <= 2^22 words are
 * rejected with CKKS_EINVAL.  No cudaMalloc / cudaFree (or any allocating routine) is
 * called; per-kernel timing is suspended during the call.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current: make that
 * first call before any stream capture (a first call on a capturing stream returns
 * CKKS_EINVAL).  Every call shares the array and leaves its
 * contents behind; nothing in it needs to start at zero (each word is written before it is
 * read), but calls that overlap on the GPU (other streams, other contexts on the same
 * device) race on it. */
int ckks_rescale_noalloc(ckks_ctx* ctx, const uint64_t* d_in, int level, uint64_t* d_out);

/* HActivation (Sec. 2.4.2; Alg. 1, activation step) as a composite polynomial ReLU:
 * y = s_k(...s_1(x)) with each stage a Chebyshev series (coefficients concatenated in
 * `coeffs`, degrees in degs[n_stages], evaluated as by ckks_eval_poly), then x * y with x
 * brought down to y's level.  With s_1..s_{k-1} normalised odd sign approximations and
 * s_k = (1 + sign approximation) / 2 this is x (1 + sign(x)) / 2.  Levels used:
 * sum_i (ceil(log2 deg_i) + 1) + 1, and one more when the stages cross from the bootstrapping
 * segment of the chain into the circuit segment (18 for degrees (15, 15, 27) from level 23). */
int ckks_eval_relu(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const double* coeffs, const int* degs,
                   int n_stages, ckks_ct* out);

/* ---- raw kernels on caller device memory ---------------------------------- */
/* In-place forward / inverse negacyclic NTT of n_limbs limbs at `dev` ([n_limbs][N]
 * uint64 device memory, residues < q); limb i uses the prime with global id
 * prime_ids[i] (q_0..q_L are 0..L, p_j is n_q + j).  Forward: out[i] =
 * sum_j a[j] psi^((2 rev(i) + 1) j), bit-reversed order. */
int ckks_ntt_forward(ckks_ctx* ctx, uint64_t* dev, int n_limbs, const int32_t* prime_ids);
int ckks_ntt_inverse(ckks_ctx* ctx, uint64_t* dev, int n_limbs, const int32_t* prime_ids);

#ifdef __cplusplus
}
#endif
#endif /* CKKS_GB300_H */
