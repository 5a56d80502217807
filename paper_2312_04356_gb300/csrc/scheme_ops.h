// Internal scheme operations (scheme.cu), used by the C ABI (capi.cpp).
#pragma once
#include "internal.h"

namespace ops {
DevBuf upload(ckks_ctx* c, const std::vector<u64>& v);
void ensure_ct(ckks_ct& ct, ckks_ctx* c, int level, int nb = 1);
ckks_ct new_ct(ckks_ctx* c, int level, double scale, int nb = 1);
ckks_ct copy_ct(const ckks_ct& a);
ckks_ct add(const ckks_ct& a, const ckks_ct& b);
ckks_ct sub(const ckks_ct& a, const ckks_ct& b);
ckks_ct mul_plain(const ckks_ct& a, const ckks_pt& p);
void mul_plain_acc(ckks_ct& o, const ckks_ct& a, const ckks_pt& p);
ckks_ct mul_int(const ckks_ct& a, long long v);
ckks_ct add_const(const ckks_ct& a, double cst);
ckks_ct imult(const ckks_ct& a);
ckks_ct rescale(const ckks_ct& a);
// rescale(mul_int(a, k)) in one pass over the limbs (identical residues)
ckks_ct rescale_mul(const ckks_ct& a, long long k);
ckks_ct mod_drop(const ckks_ct& a, int level);
ckks_ct level_down(const ckks_ct& a, int level);
ckks_ct mod_raise(const ckks_ct& a);
// per digit, the polynomial x (NTT domain, [l+1][N]) raised to Q_l u P: [ndig][next][N]; for a
// batch, nb polynomials at x + t xstride -> [nb][ndig][next][N]
DevBuf mod_up(ckks_ctx* c, const u64* x, int level, int* ndig_out, int nb = 1, size_t xstride = 0);

u64 galois_of_step(const ckks_ctx* c, long long r);
std::vector<ckks_ct> rotate_hoisted(const ckks_keys& keys, const ckks_ct& a, const std::vector<long long>& steps);
ckks_ct rotate(const ckks_keys& keys, const ckks_ct& a, long long r);
ckks_ct conjugate(const ckks_keys& keys, const ckks_ct& a);
ckks_ct mul_relin(const ckks_keys& keys, const ckks_ct& a, const ckks_ct& b);
// twice: 2 a b (the doubling folded into the rescale's tail; same residues as add(t, t))
ckks_ct mul_relin_rescale(const ckks_keys& keys, const ckks_ct& a, const ckks_ct& b, bool twice = false);
ckks_ct bsgs(const ckks_keys& keys, const ckks_ct& a, const ckks_ptset& ps, bool rescale_out = false);
ckks_ct bsgs_multi(const ckks_keys& keys, const std::vector<const ckks_ct*>& ins,
                   const std::vector<const ckks_ptset*>& pss, bool rescale_out);
ckks_ct cheb_eval(const ckks_keys& keys, const ckks_ct& x, const std::vector<double>& coeffs);
ckks_ct eval_mod(const ckks_keys& keys, const ckks_ct& x, const std::vector<double>& coeffs, int r);
ckks_ct affine(const ckks_ct& x, double alpha, double beta);
ckks_ct eval_poly(const ckks_keys& keys, const ckks_ct& x, const std::vector<double>& coeffs, bool power, double a,
                  double b);
ckks_ct eval_relu(const ckks_keys& keys, const ckks_ct& x, const std::vector<std::vector<double>>& stages);
void bootstrap(const ckks_keys& keys, const ckks_boot& bt, const ckks_ct& ct0, ckks_ct& re_out, ckks_ct& im_out);
ckks_ct stoc1(const ckks_keys& keys, const ckks_boot& bt, const ckks_ct& re, const ckks_ct& im);
ckks_ct block(const ckks_keys& keys, const ckks_boot& bt, const ckks_ptset& conv, const ckks_ct& in);
ckks_ct block_multi(const ckks_keys& keys, const ckks_boot& bt, const std::vector<const ckks_ptset*>& convs,
                    const std::vector<const ckks_ct*>& ins);
ckks_ct downsample_layer(const ckks_keys& keys, const ckks_boot& bt_in, const ckks_boot& bt_out,
                         const std::vector<const ckks_ct*>& re, const std::vector<const ckks_ct*>& im,
                         const std::vector<const ckks_ptset*>& convs);
void add_galois_key(ckks_ctx* c, ckks_keys& K, u64 g);
ckks_keys* keygen(ckks_ctx* c, const int32_t* steps, int nsteps, int want_conj);
ckks_ct encrypt(const ckks_keys& K, const ckks_pt& pt, u64 nonce);
ckks_ct encrypt_sk(const ckks_keys& K, const ckks_pt& pt, u64 nonce);
void decrypt(const ckks_keys& K, const ckks_ct& ct, ckks_pt& out);
}  // namespace ops

ckks_ctx* ctx_create(const ckks_params* P, uint64_t seed, cudaStream_t stream);
