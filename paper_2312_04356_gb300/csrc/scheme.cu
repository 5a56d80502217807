// RNS-CKKS scheme on the GPU: context, keys, encryption, key switching, rotations,
// BSGS linear maps, the fused CinS conv, Chebyshev evaluation and bootstrapping.
//
// Every ciphertext limb lives on the device in the NTT domain.  Host code only
// sequences kernels (kernels.cu) and prepares constants.  Steps follow the paper's
// Alg. 1 and the hybrid RNS-CKKS it builds on (Sec. 2.1, Sec. 2.4):
//   key switching: digits of alpha consecutive limbs; ModUp by fast base conversion
//   without correction; inner product with the key over Q_l u P; ModDown
//   (c - Conv_{P->Q}([c]_P)) P^{-1}.  Rotations are always hoisted: ModUp(c1) once,
//   then per step the automorphism is applied to the raised digits inside the inner
//   product (k_ks_inner gathers through the Galois permutation).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <set>

#include "internal.h"
#include "scheme_ops.h"

using namespace hostmath;

namespace {

enum { K_SK = 1, K_SK_SIGN = 2, K_PK_A = 3, K_PK_E = 4, K_SWK_A = 5, K_SWK_E = 6, K_ENC_U = 7, K_ENC_E0 = 8,
       K_ENC_E1 = 9, K_ENCSK_A = 10, K_ENCSK_E = 11 };

inline u64 tag(u64 kind, u64 a = 0, u64 b = 0) { return (kind << 56) | (a << 16) | b; }

template <class T>
T* dev_upload_persistent(const std::vector<T>& v) {
    T* p = nullptr;
    if (v.empty()) return nullptr;
    CUDA_CHECK(cudaMalloc((void**)&p, v.size() * sizeof(T)));
    CUDA_CHECK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

}  // namespace

namespace ops {

DevBuf upload(ckks_ctx* c, const std::vector<u64>& v) {
    DevBuf b(v.size(), c->stream);
    if (!v.empty()) CUDA_CHECK(cudaMemcpyAsync(b.ptr, v.data(), v.size() * 8, cudaMemcpyHostToDevice, c->stream));
    return b;
}

}  // namespace ops

// ============================================================ context ======
std::vector<std::vector<int>> ckks_ctx::digits(int level) const {
    std::vector<std::vector<int>> out;
    for (int d = 0; d < P.dnum; ++d) {
        int lo = d * alpha, hi = std::min((d + 1) * alpha, level + 1);
        if (lo < hi) {
            std::vector<int> g;
            for (int i = lo; i < hi; ++i) g.push_back(i);
            out.push_back(g);
        }
    }
    return out;
}

std::vector<int> ckks_ctx::ext_ids(int level) const {
    std::vector<int> v;
    for (int i = 0; i <= level; ++i) v.push_back(i);
    for (int j = 0; j < np; ++j) v.push_back(nq + j);
    return v;
}

static std::unique_ptr<ConvTab> make_conv_tab(ckks_ctx* c, const std::vector<int>& in_ids,
                                              const std::vector<int>& out_ids, const std::vector<int>& out_rows,
                                              bool exact = false) {
    auto t = std::make_unique<ConvTab>();
    t->nin = (int)in_ids.size();
    t->nout = (int)out_ids.size();
    t->in_ids = in_ids;
    t->out_ids = out_ids;
    std::vector<u64> qinv(2 * t->nin), qmod(2 * (size_t)t->nout * t->nin);
    for (int i = 0; i < t->nin; ++i) {
        u64 qi = c->mod_of[in_ids[i]];
        u64 prod = 1;
        for (int k = 0; k < t->nin; ++k)
            if (k != i) prod = mulmod(prod, c->mod_of[in_ids[k]] % qi, qi);
        qinv[i] = invmod(prod, qi);
        qinv[t->nin + i] = shoup(qinv[i], qi);
        for (int m = 0; m < t->nout; ++m) {
            u64 pm = c->mod_of[out_ids[m]];
            u64 v = 1;
            for (int k = 0; k < t->nin; ++k)
                if (k != i) v = mulmod(v, c->mod_of[in_ids[k]] % pm, pm);
            qmod[(size_t)m * t->nin + i] = v;
            qmod[(size_t)t->nout * t->nin + (size_t)m * t->nin + i] = shoup(v, pm);
        }
    }
    // N^{-1} qhat_i^{-1}: the inverse NTT that produces this conversion's inputs ends with it
    std::vector<u64> isc(2 * t->nin);
    for (int i = 0; i < t->nin; ++i) {
        const u64 qi = c->mod_of[in_ids[i]];
        isc[2 * i] = mulmod(invmod((u64)c->n % qi, qi), qinv[i], qi);
        isc[2 * i + 1] = shoup(isc[2 * i], qi);
    }
    t->d_iscale = dev_upload_persistent(isc);
    std::vector<int> ids_rows = out_ids;
    ids_rows.insert(ids_rows.end(), out_rows.begin(), out_rows.end());
    t->d_in_ids = dev_upload_persistent(in_ids);
    t->d_out_ids = dev_upload_persistent(ids_rows);
    t->d_qhat_inv = dev_upload_persistent(qinv);
    t->d_qhat_mod = dev_upload_persistent(qmod);
    {
        std::vector<u64> pm(t->nout), r24p;
        for (int m = 0; m < t->nout; ++m) pm[m] = c->mod_of[out_ids[m]];
        t->d_tcb = dev_upload_persistent(kern::conv_tc_image(qmod, pm, t->nin, t->nout, t->tc_nin2, t->tc_S,
                                                             t->tc_groups, r24p));
        if (t->d_tcb) t->d_tcr = dev_upload_persistent(r24p);
    }
    if (exact) {
        // 1/q_i = M_i 2^-(64 + b_i): the rounding term in fixed point (kern: conv_round)
        std::vector<u64> invq(2 * t->nin);
        for (int i = 0; i < t->nin; ++i) {
            const u64 qi = c->mod_of[in_ids[i]];
            int b = 63;
            while (!((qi >> b) & 1)) --b;
            invq[i] = (u64)((((unsigned __int128)1) << (64 + b)) / qi);
            invq[t->nin + i] = (u64)(b + 6);
        }
        std::vector<u64> corr(2 * t->nout);
        for (int m = 0; m < t->nout; ++m) {
            const u64 pm = c->mod_of[out_ids[m]];
            u64 v = 1;
            for (int k = 0; k < t->nin; ++k) v = mulmod(v, c->mod_of[in_ids[k]] % pm, pm);
            corr[m] = v ? pm - v : 0;
            corr[t->nout + m] = shoup(corr[m], pm);
        }
        t->d_inv_q = dev_upload_persistent(invq);
        t->d_corr = dev_upload_persistent(corr);
    }
    return t;
}

const ConvTab& ckks_ctx::modup_tab(int level, int d) {
    auto key = std::make_pair(level, d);
    auto it = modup_tabs.find(key);
    if (it != modup_tabs.end()) return *it->second;
    std::vector<int> dig = digits(level)[d];
    std::vector<int> ext = ext_ids(level);
    std::vector<int> out_ids, out_rows;
    for (int r = 0; r < (int)ext.size(); ++r) {
        if (r >= dig.front() && r <= dig.back()) continue;
        out_ids.push_back(ext[r]);
        out_rows.push_back(r);
    }
    modup_tabs[key] = make_conv_tab(this, dig, out_ids, out_rows);
    return *modup_tabs[key];
}

const ConvTab& ckks_ctx::moddown_tab(int level) {
    auto it = moddown_tabs.find(level);
    if (it != moddown_tabs.end()) return *it->second;
    std::vector<int> in_ids, out_ids, out_rows;
    for (int j = 0; j < np; ++j) in_ids.push_back(nq + j);
    for (int i = 0; i <= level; ++i) {
        out_ids.push_back(i);
        out_rows.push_back(i);
    }
    moddown_tabs[level] = make_conv_tab(this, in_ids, out_ids, out_rows);
    return *moddown_tabs[level];
}

// ModDown fused with a rescale: inputs q_l and the special primes (rows l .. l + np of the
// extended layout), outputs q_0 .. q_{l-1}
const ConvTab& ckks_ctx::mdrs_tab(int level) {
    auto it = mdrs_tabs.find(level);
    if (it != mdrs_tabs.end()) return *it->second;
    std::vector<int> in_ids, out_ids, out_rows;
    in_ids.push_back(level);
    for (int j = 0; j < np; ++j) in_ids.push_back(nq + j);
    for (int i = 0; i < level; ++i) {
        out_ids.push_back(i);
        out_rows.push_back(i);
    }
    mdrs_tabs[level] = make_conv_tab(this, in_ids, out_ids, out_rows, true);
    return *mdrs_tabs[level];
}

static void free_tab(ConvTab* t) {
    cudaFree(t->d_in_ids);
    cudaFree(t->d_out_ids);
    cudaFree(t->d_qhat_inv);
    cudaFree(t->d_qhat_mod);
    if (t->d_inv_q) cudaFree(t->d_inv_q);
    if (t->d_corr) cudaFree(t->d_corr);
    cudaFree(t->d_iscale);
}

ckks_ctx::~ckks_ctx() {
    for (int k = 0; k < NSIDE; ++k) {
        if (side_ev[k]) cudaEventDestroy(side_ev[k]);
        if (side[k]) cudaStreamDestroy(side[k]);
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
    cudaStreamSynchronize(stream);
    for (auto& kv : modup_tabs) free_tab(kv.second.get());
    for (auto& kv : moddown_tabs) free_tab(kv.second.get());
    for (auto& kv : mdrs_tabs) free_tab(kv.second.get());
    for (int* p : d_ext_ids) cudaFree(p);
    for (int* p : d_modup_off) cudaFree(p);
    for (int* p : d_modup_pid) cudaFree(p);
    for (u64* p : d_modup_iscale) cudaFree(p);
    cudaFree(d_iota);
    cudaFree(d_primes);
    cudaFree(d_tables);
    cudaFree(d_gauss);
    cudaFree(d_pinv);
    cudaFree(d_qlinv);
    cudaFree(d_pqlinv);
    cudaFree(d_pqlinv2);
    cudaFree(d_pmod);
}

static unsigned brev_host(unsigned x, int bits) {
    unsigned r = 0;
    for (int i = 0; i < bits; ++i) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

ckks_ctx* ctx_create(const ckks_params* P, uint64_t seed, cudaStream_t stream) {
    CK_CHECK(P && P->log_n >= 3 && P->log_n <= 17, CKKS_EINVAL, "log_n must be in 3..17");
    CK_CHECK(P->n_q >= 1 && P->dnum >= 1 && P->n_boot >= 0 && P->n_boot < P->n_q, CKKS_EINVAL, "bad n_q/dnum/n_boot");
    CK_CHECK(P->q0_bits <= 61 && P->p_bits <= 61 && P->scale_bits <= 61 && P->boot_bits <= 61, CKKS_EINVAL,
             "primes must stay below 2^61");
    std::unique_ptr<ckks_ctx> c(new ckks_ctx());
    c->P = *P;
    c->logn = P->log_n;
    c->n = 1 << P->log_n;
    c->nq = P->n_q;
    c->L = P->n_q - 1;
    c->alpha = (P->n_q + P->dnum - 1) / P->dnum;
    c->np = P->n_p > 0 ? P->n_p : c->alpha;
    c->nall = c->nq + c->np;
    c->n_circuit = c->L - P->n_boot;
    c->seed = seed;
    c->stream = stream;
    CK_CHECK(c->alpha <= 16 && c->np <= 16, CKKS_EINVAL, "digits and special primes are limited to 16 limbs");
    build_chain(*P, c->q, c->p, c->delta);
    c->mod_of = c->q;
    c->mod_of.insert(c->mod_of.end(), c->p.begin(), c->p.end());
    c->mods_below_2_60 = std::all_of(c->mod_of.begin(), c->mod_of.end(), [](u64 m) { return m < (1ull << 60); });
    const int n = c->n, logn = c->logn;
    // twiddle tables: per prime 2 arrays of N (value, Shoup companion) pairs
    std::vector<u64> tables((size_t)c->nall * 4 * n);
    std::vector<DevPrime> primes(c->nall);
    c->psi.resize(c->nall);
    c->mods.resize(c->nall);
    CUDA_CHECK(cudaMalloc((void**)&c->d_tables, tables.size() * sizeof(u64)));
    std::vector<u64> pw(n), ipw(n);
    for (int id = 0; id < c->nall; ++id) {
        const u64 qq = c->mod_of[id];
        const u64 psi = smallest_root_2n(qq, n);
        const u64 ipsi = invmod(psi, qq);
        c->psi[id] = psi;
        c->mods[id] = make_mod(qq);
        pw[0] = ipw[0] = 1;
        for (int e = 1; e < n; ++e) {
            pw[e] = mulmod(pw[e - 1], psi, qq);
            ipw[e] = mulmod(ipw[e - 1], ipsi, qq);
        }
        u64* base = tables.data() + (size_t)id * 4 * n;
        for (int k = 0; k < n; ++k) {
            unsigned r = brev_host(k, logn);
            base[2 * k] = pw[r];
            base[2 * k + 1] = shoup(pw[r], qq);
            base[2 * n + 2 * k] = ipw[r];
            base[2 * n + 2 * k + 1] = shoup(ipw[r], qq);
        }
        DevPrime& dp = primes[id];
        dp.m = c->mods[id];
        const u64* dbase = c->d_tables + (size_t)id * 4 * n;
        dp.tw = reinterpret_cast<const ulonglong2*>(dbase);
        dp.itw = reinterpret_cast<const ulonglong2*>(dbase + 2 * n);
        dp.n_inv = invmod((u64)n % qq, qq);
        dp.n_inv_p = shoup(dp.n_inv, qq);
        dp.r64 = (u64)(((unsigned __int128)1 << 64) % qq);
        dp.r64p = shoup(dp.r64, qq);
        dp.inv64 = (u64)((((unsigned __int128)1) << 64) / qq);
    }
    CUDA_CHECK(cudaMemcpy(c->d_tables, tables.data(), tables.size() * sizeof(u64), cudaMemcpyHostToDevice));
    c->d_primes = dev_upload_persistent(primes);
    gauss_table(P->sigma, c->gauss);
    c->d_gauss = dev_upload_persistent(std::vector<u64>(c->gauss, c->gauss + 39));
    std::vector<int> iota(c->nall);
    for (int i = 0; i < c->nall; ++i) iota[i] = i;
    c->d_iota = dev_upload_persistent(iota);
    for (int l = 0; l <= c->L; ++l) c->d_ext_ids.push_back(dev_upload_persistent(c->ext_ids(l)));
    // P^{-1} mod q_i and q_l^{-1} mod q_i (Shoup pairs)
    std::vector<u64> pinv(2 * c->nq), qlinv(2 * (size_t)c->nq * c->nq, 0);
    for (int i = 0; i < c->nq; ++i) {
        u64 pr = 1;
        for (u64 pj : c->p) pr = mulmod(pr, pj % c->q[i], c->q[i]);
        pinv[i] = invmod(pr, c->q[i]);
        pinv[c->nq + i] = shoup(pinv[i], c->q[i]);
    }
    for (int l = 1; l < c->nq; ++l)
        for (int i = 0; i < l; ++i) {
            u64 v = invmod(c->q[l] % c->q[i], c->q[i]);
            qlinv[(size_t)l * c->nq + i] = v;
            qlinv[(size_t)c->nq * c->nq + (size_t)l * c->nq + i] = shoup(v, c->q[i]);
        }
    // (P q_l)^{-1} mod q_i (i < l) and P mod q_i (Shoup pairs)
    std::vector<u64> pqlinv(2 * (size_t)c->nq * c->nq, 0), pmod(2 * c->nq);
    for (int i = 0; i < c->nq; ++i) {
        u64 pr = 1;
        for (u64 pj : c->p) pr = mulmod(pr, pj % c->q[i], c->q[i]);
        pmod[i] = pr;
        pmod[c->nq + i] = shoup(pr, c->q[i]);
    }
    std::vector<u64> pqlinv2(2 * (size_t)c->nq * c->nq, 0);
    for (int l = 1; l < c->nq; ++l)
        for (int i = 0; i < l; ++i) {
            u64 v = invmod(mulmod(pmod[i], c->q[l] % c->q[i], c->q[i]), c->q[i]);
            pqlinv[(size_t)l * c->nq + i] = v;
            pqlinv[(size_t)c->nq * c->nq + (size_t)l * c->nq + i] = shoup(v, c->q[i]);
            const u64 v2 = mulmod(v, 2, c->q[i]);
            pqlinv2[(size_t)l * c->nq + i] = v2;
            pqlinv2[(size_t)c->nq * c->nq + (size_t)l * c->nq + i] = shoup(v2, c->q[i]);
        }
    c->d_pinv = dev_upload_persistent(pinv);
    c->d_qlinv = dev_upload_persistent(qlinv);
    c->h_qlinv.assign(qlinv.begin(), qlinv.begin() + (size_t)c->nq * c->nq);
    c->d_pqlinv = dev_upload_persistent(pqlinv);
    c->d_pqlinv2 = dev_upload_persistent(pqlinv2);
    c->d_pmod = dev_upload_persistent(pmod);
    // every base-conversion table up front (no allocation later, e.g. inside stream capture)
    for (int l = 0; l <= c->L; ++l) {
        c->moddown_tab(l);
        if (l >= 1) c->mdrs_tab(l);
        std::vector<std::vector<int>> dig = c->digits(l);
        std::vector<int> ext = c->ext_ids(l), off, pid;
        const int next = (int)ext.size();
        for (int d = 0; d < (int)dig.size(); ++d) {
            c->modup_tab(l, d);
            for (int r = 0; r < next; ++r) {
                if (r >= dig[d].front() && r <= dig[d].back()) continue;
                off.push_back(d * next + r);
                pid.push_back(ext[r]);
            }
        }
        c->d_modup_off.push_back(dev_upload_persistent(off));
        c->d_modup_pid.push_back(dev_upload_persistent(pid));
        c->modup_nrows.push_back((int)off.size());
        // the final factor of the inverse NTT of a ModUp input: row r of digit d gets that
        // digit's N^{-1} qhat^{-1}
        std::vector<u64> isc;
        for (int d = 0; d < (int)dig.size(); ++d) {
            std::vector<u64> h(2 * dig[d].size());
            CUDA_CHECK(cudaMemcpy(h.data(), c->modup_tab(l, d).d_iscale, h.size() * 8, cudaMemcpyDeviceToHost));
            isc.insert(isc.end(), h.begin(), h.end());
        }
        c->d_modup_iscale.push_back(dev_upload_persistent(isc));
    }
    cudaMemPool_t pool;
    int dev = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    return c.release();
}

// ============================================================ helpers ======
namespace ops {

void ensure_ct(ckks_ct& ct, ckks_ctx* c, int level, int nb) {
    ct.ctx = c;
    size_t need = (size_t)nb * 2 * (size_t)(level + 1) * c->n;
    if (ct.buf.words < need || ct.buf.ptr == nullptr) ct.buf = DevBuf(need, c->stream);
    ct.level = level;
    ct.nb = nb;
}

ckks_ct new_ct(ckks_ctx* c, int level, double scale, int nb) {
    ckks_ct ct;
    ensure_ct(ct, c, level, nb);
    ct.scale = scale;
    return ct;
}

ckks_ct copy_ct(const ckks_ct& a) {
    ckks_ct o = new_ct(a.ctx, a.level, a.scale, a.nb);
    CUDA_CHECK(cudaMemcpyAsync(o.buf.ptr, a.buf.ptr, a.nb * a.cstride() * 8, cudaMemcpyDeviceToDevice,
                               a.ctx->stream));
    return o;
}

static void check_same(const ckks_ct& a, const ckks_ct& b) {
    CK_CHECK(a.nb == b.nb, CKKS_EINVAL, "batch sizes differ");
    CK_CHECK(a.level == b.level, CKKS_EINVAL, "ciphertext levels differ");
    CK_CHECK(fabs(a.scale - b.scale) <= ldexp(1.0, -30) * fabs(a.scale), CKKS_EINVAL, "ciphertext scales differ");
}

ckks_ct add(const ckks_ct& a, const ckks_ct& b) {
    check_same(a, b);
    ckks_ctx* c = a.ctx;
    ckks_ct o = new_ct(c, a.level, a.scale, a.nb);
    kern::add(c, a.buf.ptr, b.buf.ptr, o.buf.ptr, 2 * (a.level + 1) * a.nb, c->d_iota, a.level + 1);
    return o;
}

ckks_ct sub(const ckks_ct& a, const ckks_ct& b) {
    check_same(a, b);
    ckks_ctx* c = a.ctx;
    ckks_ct o = new_ct(c, a.level, a.scale, a.nb);
    kern::sub(c, a.buf.ptr, b.buf.ptr, o.buf.ptr, 2 * (a.level + 1) * a.nb, c->d_iota, a.level + 1);
    return o;
}

ckks_ct mul_plain(const ckks_ct& a, const ckks_pt& p) {
    CK_CHECK(p.level == a.level, CKKS_EINVAL, "plaintext level differs from the ciphertext level");
    ckks_ctx* c = a.ctx;
    c->ops["pmult"]++;
    ckks_ct o = new_ct(c, a.level, a.scale * p.scale, a.nb);
    const int nl = a.level + 1;
    // c0 and c1 of every ciphertext of the batch times the one plaintext, one launch
    kern::mul(c, a.buf.ptr, p.buf.ptr, o.buf.ptr, 2 * nl * a.nb, c->d_iota, nl, nl);
    return o;
}

// o += a * p (both polynomials)
void mul_plain_acc(ckks_ct& o, const ckks_ct& a, const ckks_pt& p) {
    CK_CHECK(p.level == a.level && o.level == a.level, CKKS_EINVAL, "level mismatch in multiply-accumulate");
    CK_CHECK(a.nb == 1 && o.nb == 1, CKKS_EINVAL, "multiply-accumulate takes single ciphertexts");
    ckks_ctx* c = a.ctx;
    c->ops["pmult"]++;
    const int nl = a.level + 1;
    kern::mul_acc(c, a.c0(), p.buf.ptr, o.c0(), nl, c->d_iota, nl);
    kern::mul_acc(c, a.c1(), p.buf.ptr, o.c1(), nl, c->d_iota, nl);
}

ckks_ct mul_int(const ckks_ct& a, long long v) {
    ckks_ctx* c = a.ctx;
    const int nl = a.level + 1;
    ScalarVec sv;
    for (int i = 0; i < nl; ++i) {
        sv.v[i] = from_signed(v, c->q[i]);
        sv.vp[i] = shoup(sv.v[i], c->q[i]);
    }
    ckks_ct o = new_ct(c, a.level, a.scale, a.nb);
    kern::mul_scalar_v(c, a.buf.ptr, sv, o.buf.ptr, 2 * nl * a.nb, c->d_iota, nl);
    return o;
}

ckks_ct add_const(const ckks_ct& a, double cst) {
    ckks_ctx* c = a.ctx;
    const int nl = a.level + 1;
    long long v = llround_away(cst * a.scale);
    ScalarVec sv;
    for (int i = 0; i < nl; ++i) sv.v[i] = from_signed(v, c->q[i]);
    ckks_ct o = copy_ct(a);
    kern::add_scalar_v(c, o.c0(), sv, nl * a.nb, c->d_iota, nl, a.cstride());    // c0 of each ciphertext
    return o;
}

ckks_ct imult(const ckks_ct& a) {
    ckks_ctx* c = a.ctx;
    ckks_ct o = new_ct(c, a.level, a.scale, a.nb);
    kern::imult(c, a.buf.ptr, o.buf.ptr, 2 * (a.level + 1) * a.nb, c->d_iota, a.level + 1);
    return o;
}

// rescale(mul_int(a, k)) without materialising a k: the dropped limbs are scaled by k while
// they are copied out, and the tail computes a_i (k q_l^{-1}) - lift_i q_l^{-1} (the same
// residues as (k a_i - lift_i) q_l^{-1}); like rescale(mul_int(a, k)) the scale becomes
// a.scale / q_l (callers track the integer factor themselves).
ckks_ct rescale_mul(const ckks_ct& a, long long k) {
    ckks_ctx* c = a.ctx;
    const int l = a.level;
    CK_CHECK(l >= 1, CKKS_ELEVEL, "cannot rescale a level-0 ciphertext");
    CK_CHECK(l <= ScalarVec::MAX, CKKS_EINVAL, "too many limbs for a by-value scalar vector");
    c->ops["rescale"]++;
    const size_t n = c->n;
    // k times the last limb of every polynomial (c0, c1 of each ciphertext: 2 nb rows (l + 1) N
    // apart), to the coefficient domain; then its centred lift to the other l primes, back to
    // the NTT domain
    const int np_ = 2 * a.nb;
    DevBuf last((size_t)np_ * n, c->stream);
    kern::ntt_inverse_from(c, a.c0() + (size_t)l * n, (size_t)(l + 1) * n, last.ptr, np_, c->d_iota + l, 1, n,
                           nullptr, from_signed(k, c->q[l]), l);
    DevBuf lift((size_t)np_ * l * n, c->stream);
    kern::lift_centred(c, last.ptr, l, lift.ptr, np_ * l, c->d_iota, l, n);     // every polynomial
    kern::ntt_forward(c, lift.ptr, np_ * l, c->d_iota, l);
    ckks_ct o = new_ct(c, l - 1, a.scale / (double)c->q[l], a.nb);
    ScalarVec s1;
    for (int i = 0; i < l; ++i) {
        s1.v[i] = mulmod(from_signed(k, c->q[i]), c->h_qlinv[(size_t)l * c->nq + i], c->q[i]);
        s1.vp[i] = shoup(s1.v[i], c->q[i]);
    }
    const u64* s2 = c->d_qlinv + (size_t)l * c->nq;
    const u64* s2p = c->d_qlinv + (size_t)c->nq * c->nq + (size_t)l * c->nq;
    kern::sub_mul2_scalar(c, a.c0(), lift.ptr, s1, s2, s2p, o.c0(), np_ * l, c->d_iota, l, (size_t)(l + 1) * n);
    return o;
}

ckks_ct rescale(const ckks_ct& a) { return rescale_mul(a, 1); }

ckks_ct mod_drop(const ckks_ct& a, int level) {
    CK_CHECK(level >= 0 && level <= a.level, CKKS_EINVAL, "mod_drop to a higher level");
    ckks_ctx* c = a.ctx;
    ckks_ct o = new_ct(c, level, a.scale, a.nb);
    const size_t bytes = (size_t)(level + 1) * c->n * 8;
    // the first level + 1 limbs of every polynomial: 2 nb rows of `bytes`
    CUDA_CHECK(cudaMemcpy2DAsync(o.c0(), bytes, a.c0(), (size_t)(a.level + 1) * c->n * 8, bytes, 2 * a.nb,
                                 cudaMemcpyDeviceToDevice, c->stream));
    return o;
}

ckks_ct level_down(const ckks_ct& a, int level) {
    ckks_ctx* c = a.ctx;
    CK_CHECK(level >= 0 && level <= a.level, CKKS_EINVAL, "level_down to a higher level");
    if (level == a.level) return copy_ct(a);
    ckks_ct x;
    const ckks_ct* cur = &a;
    while (cur->level > level) {
        const int l = cur->level;
        long long k = llround_away((c->delta[l - 1] * (double)c->q[l]) / cur->scale);
        ckks_ct t = rescale_mul(*cur, k);
        t.scale = c->delta[l - 1];
        x = std::move(t);
        cur = &x;
    }
    return x;
}

ckks_ct mod_raise(const ckks_ct& a) {
    ckks_ctx* c = a.ctx;
    CK_CHECK(a.level == 0, CKKS_EINVAL, "ModRaise needs a level-0 ciphertext");
    const size_t n = c->n;
    const int np_ = 2 * a.nb;                        // a level-0 batch is np_ consecutive limbs
    DevBuf coef((size_t)np_ * n, c->stream);
    kern::ntt_inverse_from(c, a.c0(), n, coef.ptr, np_, c->d_iota, 1, n, nullptr);
    ckks_ct o = new_ct(c, c->L, a.scale, a.nb);
    kern::lift_centred(c, coef.ptr, 0, o.buf.ptr, np_ * c->nq, c->d_iota, c->nq, n);   // row k from source k / nq
    kern::ntt_forward(c, o.buf.ptr, np_ * c->nq, c->d_iota, c->nq);
    return o;
}

// ------------------------------------------------------- key switching -----
// D: [ndig][next][N], NTT domain; for a batch, x of ciphertext t at x + t xstride and D
// [nb][ndig][next][N]
DevBuf mod_up(ckks_ctx* c, const u64* x, int level, int* ndig_out, int nb, size_t xstride) {
    const size_t n = c->n;
    const int nl = level + 1;
    const int next = nl + c->np;
    std::vector<std::vector<int>> dig = c->digits(level);
    const int ndig = (int)dig.size();
    const size_t dstr = (size_t)ndig * next * n;     // words per ciphertext of D
    if (xstride == 0) xstride = (size_t)nl * n;
    DevBuf coef((size_t)nb * nl * n, c->stream);
    kern::ntt_inverse_from(c, x, xstride, coef.ptr, nb * nl, c->d_iota, nl, (size_t)nl * n,
                           c->d_modup_iscale[level]);   // prescaled
    DevBuf D((size_t)nb * dstr, c->stream);
    const int* ext = c->d_ext_ids[level];
    kern::ConvJobs jobs;
    jobs.n = 0;
    for (int d = 0; d < ndig; ++d)
        kern::add_conv_job(jobs, c->modup_tab(level, d), coef.ptr + (size_t)dig[d].front() * n,
                           D.ptr + (size_t)d * next * n, (size_t)nl * n, dstr, true);
    kern::base_convert_jobs(c, jobs, nb);
    for (int d = 0; d < ndig; ++d) {
        u64* Dd = D.ptr + (size_t)d * next * n;
        const int lo = dig[d].front(), hi = dig[d].back() + 1;
        CUDA_CHECK(cudaMemcpy2DAsync(Dd + (size_t)lo * n, dstr * 8, x + (size_t)lo * n, xstride * 8,
                                     (size_t)(hi - lo) * n * 8, nb, cudaMemcpyDeviceToDevice, c->stream));
        if (c->logn != 16) {
            if (lo > 0) kern::ntt_forward(c, Dd, nb * lo, ext, lo, dstr);
            if (next > hi) kern::ntt_forward(c, Dd + (size_t)hi * n, nb * (next - hi), ext + hi, next - hi, dstr);
        }
    }
    if (c->logn == 16)   // every converted row of every digit of every ciphertext in one launch
        kern::ntt_forward_list(c, D.ptr, c->modup_nrows[level], c->d_modup_off[level], c->d_modup_pid[level], nb,
                               dstr);
    *ndig_out = ndig;
    return D;
}

// inner product with switching key `code` (automorphism g applied to D on the fly) over
// Q_l u P: acc [2][next][N], NTT domain; `accumulate` adds to what acc holds.  With x0, the
// first x0rows rows of acc's first half also receive s x0(sigma_g) (s null: x0(sigma_g)), the
// automorphed c0 term of a rotation, in the same kernel.
// For a batch of nb ciphertexts: D [nb][ndig][next][N], acc [nb][2][next][N], x0 / x1 of ciphertext t
// at + t xstr; the key is read once for the batch.
void key_switch_inner(ckks_ctx* c, const ckks_keys& keys, const u64* D, int ndig, int level, u64 code, u64 g,
                      u64* acc, bool accumulate, const u64* x0 = nullptr, int x0rows = 0, const u64* s = nullptr,
                      const u64* sp = nullptr, const u64* x1 = nullptr, int nb = 1, size_t xstr = 0) {
    auto it = keys.swk.find(code);
    CK_CHECK(it != keys.swk.end(), CKKS_ENOKEY, "missing switching key (code " + std::to_string(code) + ")");
    const SwitchKey& k = *it->second;
    c->ops["keyswitch"]++;
    const size_t next = (size_t)level + 1 + c->np;
    kern::KsBatch bt;
    bt.nb = nb;
    bt.dstr = (size_t)ndig * next * c->n;
    bt.ostr = 2 * next * c->n;
    bt.xstr = xstr;
    kern::ks_inner(c, D, ndig, (int)next, c->d_ext_ids[level], k.b.ptr, k.a.ptr, acc, acc + next * c->n, g,
                   accumulate, x0, x0rows, s, sp, x1, bt);
}

// ModDown fused with the rescale after it: both halves of acc (Q_l u P, NTT domain) divided
// by P q_l, (acc - Conv_{q_l, P -> Q_{l-1}}(acc)) (P q_l)^{-1}; out [2][l][N].  A batch: acc
// [nb][2][next][N] -> out [nb][2][l][N] (every polynomial of the batch in each launch).
void mod_down_rescale(ckks_ctx* c, u64* acc, int level, u64* out, bool twice, int nb = 1) {
    CK_CHECK(level >= 1, CKKS_ELEVEL, "cannot rescale a level-0 ciphertext");
    c->ops["rescale"]++;
    const size_t n = c->n;
    const int l = level, np1 = c->np + 1, npoly = 2 * nb;
    const size_t next = (size_t)l + 1 + c->np;
    const int* pid = c->d_ext_ids[level] + l;      // q_l, then the special primes
    const ConvTab& tab_c = c->mdrs_tab(l);
    kern::ntt_inverse(c, acc + (size_t)l * n, npoly * np1, pid, np1, next * n, tab_c.d_iscale);
    DevBuf conv((size_t)npoly * l * n, c->stream);
    kern::base_convert(c, tab_c, acc + (size_t)l * n, n, conv.ptr, n, npoly, next * n, (size_t)l * n, true);
    kern::ntt_forward(c, conv.ptr, npoly * l, c->d_iota, l);
    const u64* tab = twice ? c->d_pqlinv2 : c->d_pqlinv;     // twice: 2 x the result, same pass
    const u64* s = tab + (size_t)l * c->nq;
    const u64* sp = tab + (size_t)c->nq * c->nq + (size_t)l * c->nq;
    kern::sub_mul_scalar(c, acc, conv.ptr, s, sp, out, npoly * l, c->d_iota, l, next * n);
}

// acc (Q_l u P) += P x on the Q rows, x [nb][2][l+1][N], acc [nb][2][next][N]
static void lift_p(ckks_ctx* c, const u64* x, u64* acc, int level, int nb = 1) {
    const int nl = level + 1;
    const size_t next = (size_t)nl + c->np;
    kern::mul_scalar_acc(c, x, c->d_pmod, c->d_pmod + c->nq, acc, 2 * nl * nb, c->d_iota, nl, next * c->n);
}

// ModDown of both halves of acc: [nb][2][next][N] -> out [nb][2][l+1][N]
static void mod_down(ckks_ctx* c, u64* acc, int level, u64* out, int nb = 1) {
    const size_t n = c->n;
    const int nl = level + 1, npoly = 2 * nb;
    const int next = nl + c->np;
    const int* pid = c->d_ext_ids[level] + nl;
    const ConvTab& tab_c = c->moddown_tab(level);
    kern::ntt_inverse(c, acc + (size_t)nl * n, npoly * c->np, pid, c->np, (size_t)next * n, tab_c.d_iscale);
    DevBuf conv((size_t)npoly * nl * n, c->stream);
    kern::base_convert(c, tab_c, acc + (size_t)nl * n, n, conv.ptr, n, npoly, (size_t)next * n, (size_t)nl * n,
                       true);
    kern::ntt_forward(c, conv.ptr, npoly * nl, c->d_iota, nl);
    kern::sub_mul_scalar(c, acc, conv.ptr, c->d_pinv, c->d_pinv + c->nq, out, npoly * nl, c->d_iota, nl,
                         (size_t)next * n);
}

u64 galois_of_step(const ckks_ctx* c, long long r) {
    const long long m = c->n / 2;
    r %= m;
    if (r < 0) r += m;
    return powmod(5, (u64)r, 2ULL * c->n);
}

// rot_g(a) for every ciphertext of a: the key switch of the automorphed raised digits D of c1 with
// P c0(sigma_g) added on the Q rows in the same kernel, then ModDown: ModDown(P x + k) = x +
// ModDown(k) exactly (P x vanishes on the P rows), so this is automorph(c0) + ModDown(k) in
// fewer passes.
static ckks_ct switch_galois(const ckks_keys& keys, const ckks_ct& a, const u64* D, int ndig, u64 g) {
    ckks_ctx* c = a.ctx;
    const int l = a.level, nl = l + 1;
    DevBuf acc((size_t)a.nb * 2 * ((size_t)nl + c->np) * c->n, c->stream);
    key_switch_inner(c, keys, D, ndig, l, g, g, acc.ptr, false, a.c0(), nl, c->d_pmod, c->d_pmod + c->nq, nullptr,
                     a.nb, a.cstride());
    ckks_ct o = new_ct(c, l, a.scale, a.nb);
    mod_down(c, acc.ptr, l, o.buf.ptr, a.nb);
    return o;
}

std::vector<ckks_ct> rotate_hoisted(const ckks_keys& keys, const ckks_ct& a, const std::vector<long long>& steps) {
    ckks_ctx* c = a.ctx;
    const int l = a.level;
    std::vector<ckks_ct> outs;
    DevBuf D;
    int ndig = 0;
    for (long long r : steps) {
        const u64 g = galois_of_step(c, r);
        if (g == 1) {
            outs.push_back(copy_ct(a));
            continue;
        }
        if (!D.ptr) D = mod_up(c, a.c1(), l, &ndig, a.nb, a.cstride());
        c->ops["hrot"]++;
        outs.push_back(switch_galois(keys, a, D.ptr, ndig, g));
    }
    return outs;
}

ckks_ct rotate(const ckks_keys& keys, const ckks_ct& a, long long r) {
    std::vector<ckks_ct> v = rotate_hoisted(keys, a, {r});
    return std::move(v[0]);
}

ckks_ct conjugate(const ckks_keys& keys, const ckks_ct& a) {
    ckks_ctx* c = a.ctx;
    int ndig = 0;
    DevBuf D = mod_up(c, a.c1(), a.level, &ndig, a.nb, a.cstride());
    return switch_galois(keys, a, D.ptr, ndig, 2ULL * c->n - 1);
}

// tensor product of a batch: d [nb][3][l+1][N] (d0, d1, d2 of each ciphertext)
static DevBuf tensor_batch(const ckks_ct& a, const ckks_ct& b) {
    ckks_ctx* c = a.ctx;
    const size_t nl = a.level + 1, n = c->n;
    DevBuf d((size_t)a.nb * 3 * nl * n, c->stream);
    kern::tensor(c, a.buf.ptr, b.buf.ptr, d.ptr, d.ptr + 2 * nl * n, (int)nl, c->d_iota, a.nb, a.cstride(),
                 3 * nl * n, 3 * nl * n);
    return d;
}

ckks_ct mul_relin(const ckks_keys& keys, const ckks_ct& a, const ckks_ct& b) {
    ckks_ctx* c = a.ctx;
    CK_CHECK(a.level == b.level && a.nb == b.nb, CKKS_EINVAL, "HMult operands at different levels");
    c->ops["hmult"]++;
    const int l = a.level, nl = l + 1;
    const size_t n = c->n, ds = 3 * (size_t)nl * n;
    DevBuf d = tensor_batch(a, b);
    int ndig = 0;
    DevBuf D = mod_up(c, d.ptr + 2 * (size_t)nl * n, l, &ndig, a.nb, ds);
    DevBuf acc((size_t)a.nb * 2 * ((size_t)nl + c->np) * n, c->stream);
    // relinearisation key switch with P d0, P d1 added on the Q rows in the same kernel; then
    // ModDown (= (d0, d1) + ModDown(k), see switch_galois)
    key_switch_inner(c, keys, D.ptr, ndig, l, 0, 1, acc.ptr, false, d.ptr, nl, c->d_pmod, c->d_pmod + c->nq,
                     d.ptr + (size_t)nl * n, a.nb, ds);
    ckks_ct o = new_ct(c, l, a.scale * b.scale, a.nb);
    mod_down(c, acc.ptr, l, o.buf.ptr, a.nb);
    return o;
}

// HMult, relinearisation and rescale: (d0, d1) + keyswitch(d2) kept over Q_l u P and
// divided by P q_l at once (the relinearisation's ModDown fused with the rescale)
ckks_ct mul_relin_rescale(const ckks_keys& keys, const ckks_ct& a, const ckks_ct& b, bool twice) {
    ckks_ctx* c = a.ctx;
    CK_CHECK(a.level == b.level && a.nb == b.nb, CKKS_EINVAL, "HMult operands at different levels");
    CK_CHECK(a.level >= 1, CKKS_ELEVEL, "cannot rescale a level-0 ciphertext");
    c->ops["hmult"]++;
    const int l = a.level, nl = l + 1;
    const size_t n = c->n, ds = 3 * (size_t)nl * n;
    DevBuf d = tensor_batch(a, b);                 // d0, d1, d2 of each ciphertext
    int ndig = 0;
    DevBuf D = mod_up(c, d.ptr + 2 * (size_t)nl * n, l, &ndig, a.nb, ds);
    DevBuf acc((size_t)a.nb * 2 * ((size_t)nl + c->np) * n, c->stream);
    // relinearisation key switch with P d0, P d1 added on the Q rows in the same kernel
    key_switch_inner(c, keys, D.ptr, ndig, l, 0, 1, acc.ptr, false, d.ptr, nl, c->d_pmod, c->d_pmod + c->nq,
                     d.ptr + (size_t)nl * n, a.nb, ds);
    ckks_ct o = new_ct(c, l - 1, a.scale * b.scale / (double)c->q[l], a.nb);
    mod_down_rescale(c, acc.ptr, l, o.buf.ptr, twice, a.nb);
    return o;
}

// ---------------------------------------------------------------- BSGS -----
// ModDown of one polynomial x over Q_l u P (NTT domain; its P rows are consumed): out [l+1][N];
// for a batch, nb polynomials at x + t xstride -> out [nb][l+1][N]
static void mod_down_poly(ckks_ctx* c, u64* x, int level, u64* out, int nb = 1, size_t xstride = 0) {
    const size_t n = c->n;
    const int nl = level + 1;
    if (xstride == 0) xstride = ((size_t)nl + c->np) * n;
    const ConvTab& tab_c = c->moddown_tab(level);
    kern::ntt_inverse(c, x + (size_t)nl * n, nb * c->np, c->d_ext_ids[level] + nl, c->np, xstride, tab_c.d_iscale);
    DevBuf conv((size_t)nb * nl * n, c->stream);
    kern::base_convert(c, tab_c, x + (size_t)nl * n, n, conv.ptr, n, nb, xstride, (size_t)nl * n, true);
    kern::ntt_forward(c, conv.ptr, nb * nl, c->d_iota, nl);
    kern::sub_mul_scalar(c, x, conv.ptr, c->d_pinv, c->d_pinv + c->nq, out, nb * nl, c->d_iota, nl, xstride);
}

// rot_r(a) for every r in steps kept over Q_l u P before ModDown (double hoisting), each
// [2][l+1+np][N]: (P automorph(c0) + u0, u1), u the key switch of the automorphed ModUp
// digits of c1 (one ModUp for all steps); r = 0 gives (P c0, P c1).
static std::vector<DevBuf> rotate_hoisted_ext(const ckks_keys& keys, const ckks_ct& a,
                                              const std::vector<long long>& steps) {
    ckks_ctx* c = a.ctx;
    const int l = a.level, nl = l + 1;
    const size_t n = c->n, next = (size_t)nl + c->np;
    std::vector<DevBuf> outs;
    DevBuf D;
    int ndig = 0;
    for (long long r : steps) {
        const u64 g = galois_of_step(c, r);
        DevBuf o((size_t)a.nb * 2 * next * n, c->stream);      // [nb][2][next][N]
        if (g == 1) {
            CUDA_CHECK(cudaMemsetAsync(o.ptr, 0, (size_t)a.nb * 2 * next * n * 8, c->stream));
            lift_p(c, a.buf.ptr, o.ptr, l, a.nb);
        } else {
            if (!D.ptr) D = mod_up(c, a.c1(), l, &ndig, a.nb, a.cstride());
            c->ops["hrot"]++;
            key_switch_inner(c, keys, D.ptr, ndig, l, g, g, o.ptr, false, a.c0(), nl, c->d_pmod, c->d_pmod + c->nq,
                             nullptr, a.nb, a.cstride());
        }
        outs.push_back(std::move(o));
    }
    return outs;
}

// side streams for independent work inside one operation (created on first use)
static void ensure_side_streams(ckks_ctx* c) {
    if (c->fork_ev) return;
    CUDA_CHECK(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
    for (int k = 0; k < ckks_ctx::NSIDE; ++k) {
        CUDA_CHECK(cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking));
        CUDA_CHECK(cudaEventCreateWithFlags(&c->side_ev[k], cudaEventDisableTiming));
    }
}
// puts the context's stream back when a forked section ends (also on an exception)
struct StreamRestore {
    ckks_ctx* c;
    cudaStream_t s;
    ~StreamRestore() { c->stream = s; }
};

// sum over inputs t and giant steps g of rot_{R_g}(sum_b pt_{g,b} (*) rot_{step b}(in_t)),
// double hoisted: baby steps stay over Q_l u P (one ModUp per input, no ModDown), the
// diagonals are over Q_l u P, and the inner sums of all inputs with the same giant step are
// added there.  A giant step with R != 0 brings only c1 down (ModDown), raises and
// key-switches it; its c0 is automorphed over Q_l u P.  Everything is summed over Q_l u P
// and brought down once: ModDown, or ModDown fused with the rescale when rescale_out is set.
ckks_ct bsgs_multi(const ckks_keys& keys, const std::vector<const ckks_ct*>& ins,
                   const std::vector<const ckks_ptset*>& pss, bool rescale_out) {
    ckks_ctx* c = ins[0]->ctx;
    const int l = ins[0]->level, nl = l + 1;
    const int nb = ins[0]->nb;                       // a batch: every sum below is [nb][2][next][N]
    const size_t n = c->n, next = (size_t)nl + c->np, es = 2 * next * n;
    const long long m = c->n / 2;
    const int* ext = c->d_ext_ids[l];
    const ckks_ptset& p0 = *pss[0];
    for (const ckks_ct* a : ins) CK_CHECK(a->nb == nb, CKKS_EINVAL, "the inputs of one HMatmul differ in batch size");
    for (const ckks_ptset* ps : pss)
        CK_CHECK(ps->a0 == p0.a0 && ps->step == p0.step && ps->B == p0.B && ps->G() == p0.G(), CKKS_EINVAL,
                 "the plaintext sets of one HMatmul must share their BSGS geometry");
    std::map<int, DevBuf> inner;
    double scale = 0;
    for (size_t t = 0; t < ins.size(); ++t) {
        const ckks_ct& a = *ins[t];
        const ckks_ptset& ps = *pss[t];
        CK_CHECK(a.level == ps.level && a.level == l, CKKS_EINVAL, "ciphertext level differs from the plaintext set's");
        CK_CHECK(!ps.pts.empty(), CKKS_EINVAL, "empty plaintext set");
        std::set<int> used;
        for (const auto& kv : ps.pts) used.insert(kv.first.second);
        std::vector<int> used_b(used.begin(), used.end());
        std::vector<long long> steps;
        for (int b : used_b) steps.push_back(((long long)ps.step * b) % m);
        // giant steps with at least one non-zero diagonal for this input
        std::vector<int> gs;
        for (int g = 0; g < ps.G(); ++g)
            for (int b = 0; b < ps.B; ++b)
                if (ps.pts.count(std::make_pair(g, b))) {
                    gs.push_back(g);
                    break;
                }
        if ((int)used_b.size() <= kern::BsgsFused::MAXB && (int)gs.size() <= kern::BsgsFused::MAXG &&
            c->digits(l).size() <= 4) {
            // babies and inner sums in one kernel: the baby rotations are never stored
            DevBuf D;
            int ndig = 1;
            bool any_rot = false;
            for (long long r : steps) any_rot = any_rot || r != 0;
            if (any_rot) D = mod_up(c, a.c1(), l, &ndig, nb, a.cstride());
            kern::BsgsFused T;
            T.nb = (int)used_b.size();
            T.ng = (int)gs.size();
            T.ndig = ndig;
            T.acc = 0;
            for (int i = 0; i < T.nb; ++i) {
                if (steps[i] == 0) {
                    T.kb[i] = T.ka[i] = nullptr;
                    T.gal[i] = 1;
                    continue;
                }
                const u64 gal = galois_of_step(c, steps[i]);
                auto kt = keys.swk.find(gal);
                CK_CHECK(kt != keys.swk.end(), CKKS_ENOKEY, "missing switching key (code " + std::to_string(gal) + ")");
                T.kb[i] = kt->second->b.ptr;
                T.ka[i] = kt->second->a.ptr;
                T.gal[i] = gal;
                c->ops["hrot"]++;
                c->ops["keyswitch"]++;
            }
            for (int q = 0; q < T.ng; ++q) {
                const int g = gs[q];
                for (int i = 0; i < T.nb; ++i) {
                    auto it = ps.pts.find(std::make_pair(g, used_b[i]));
                    if (it == ps.pts.end()) {
                        T.p[q][i] = nullptr;
                        continue;
                    }
                    CK_CHECK(it->second->ext, CKKS_EINVAL, "BSGS diagonals must be over Q_l u P");
                    T.p[q][i] = it->second->buf.ptr;
                    scale = a.scale * it->second->scale;
                    c->ops["pmult"]++;
                }
                auto it = inner.find(g);
                if (it == inner.end()) it = inner.emplace(g, DevBuf(nb * es, c->stream)).first;
                else T.acc |= 1u << q;
                T.o[q] = it->second.ptr;
            }
            kern::KsBatch bt;
            bt.nb = nb;
            bt.dstr = (size_t)ndig * next * n;
            bt.xstr = a.cstride();
            bt.ostr = es;
            kern::bsgs_fused(c, T, D.ptr, a.c0(), a.c1(), nl, (int)next, ext, c->d_pmod, c->d_pmod + c->nq, bt);
            continue;
        }
        std::vector<DevBuf> baby = rotate_hoisted_ext(keys, a, steps);
        // otherwise: the babies stored, then the inner sums in chunks of up to MAXG giant steps
        // (one pass over the babies per chunk)
        for (size_t k0 = 0; k0 < gs.size(); k0 += kern::BsgsGiants::MAXG) {
            kern::BsgsGiants T;
            T.nb = (int)used_b.size();
            T.ng = (int)std::min(gs.size() - k0, (size_t)kern::BsgsGiants::MAXG);
            T.acc = 0;
            CK_CHECK(T.nb <= kern::BsgsGiants::MAXB, CKKS_EINVAL, "more than 32 baby steps per giant step");
            for (int i = 0; i < T.nb; ++i) T.a[i] = baby[i].ptr;
            for (int q = 0; q < T.ng; ++q) {
                const int g = gs[k0 + q];
                for (int i = 0; i < T.nb; ++i) {
                    auto it = ps.pts.find(std::make_pair(g, used_b[i]));
                    if (it == ps.pts.end()) {
                        T.p[q][i] = nullptr;
                        continue;
                    }
                    CK_CHECK(it->second->ext, CKKS_EINVAL, "BSGS diagonals must be over Q_l u P");
                    T.p[q][i] = it->second->buf.ptr;
                    scale = a.scale * it->second->scale;
                    c->ops["pmult"]++;
                }
                auto it = inner.find(g);
                if (it == inner.end()) it = inner.emplace(g, DevBuf(nb * es, c->stream)).first;
                else T.acc |= 1u << q;
                T.o[q] = it->second.ptr;
            }
            kern::KsBatch bt;
            bt.nb = nb;
            bt.dstr = es;
            bt.ostr = es;
            kern::bsgs_inner_giants(c, T, (int)next, ext, bt);
        }
    }
    CK_CHECK(!inner.empty(), CKKS_EINVAL, "empty plaintext set");
    DevBuf acc;
    bool have_acc = false;
    // giant steps with R != 0 are independent key switches: with two or more, each runs on a
    // side stream into its own sum (its temporaries live on that stream), and the sums are
    // added on the context's stream after it has waited for all of them
    std::vector<std::pair<long long, u64*>> rot_giants;
    for (auto& kv : inner) {
        const long long R = (((long long)p0.a0 + (long long)p0.step * kv.first * p0.B) % m + m) % m;
        if (R) rot_giants.emplace_back(R, kv.second.ptr);
    }
    if (c->use_side_streams() && rot_giants.size() >= 2) {
        ensure_side_streams(c);
        std::vector<DevBuf> sums;
        for (size_t k = 0; k < rot_giants.size(); ++k) sums.emplace_back(nb * es, c->stream);
        const cudaStream_t main_stream = c->stream;
        StreamRestore restore{c, main_stream};
        CUDA_CHECK(cudaEventRecord(c->fork_ev, main_stream));
        const int nside = std::min((int)rot_giants.size(), ckks_ctx::NSIDE);
        for (int k = 0; k < nside; ++k) CUDA_CHECK(cudaStreamWaitEvent(c->side[k], c->fork_ev, 0));
        for (size_t k = 0; k < rot_giants.size(); ++k) {
            c->stream = c->side[k % ckks_ctx::NSIDE];
            const u64 gal = galois_of_step(c, rot_giants[k].first);
            u64* x = rot_giants[k].second;
            c->ops["hrot"]++;
            DevBuf c1q((size_t)nb * nl * n, c->stream);
            mod_down_poly(c, x + next * n, l, c1q.ptr, nb, es);
            int ndig = 0;
            DevBuf D = mod_up(c, c1q.ptr, l, &ndig, nb, (size_t)nl * n);
            key_switch_inner(c, keys, D.ptr, ndig, l, gal, gal, sums[k].ptr, false, x, (int)next, nullptr, nullptr,
                             nullptr, nb, es);
        }
        for (int k = 0; k < nside; ++k) {
            CUDA_CHECK(cudaEventRecord(c->side_ev[k], c->side[k]));
            CUDA_CHECK(cudaStreamWaitEvent(main_stream, c->side_ev[k], 0));
        }
        c->stream = main_stream;
        for (auto& kv : inner) {
            const long long R = (((long long)p0.a0 + (long long)p0.step * kv.first * p0.B) % m + m) % m;
            if (R) continue;
            acc = std::move(kv.second);
            have_acc = true;
        }
        for (size_t k = 0; k < sums.size(); ++k) {
            if (!have_acc) {
                acc = std::move(sums[k]);
                have_acc = true;
            } else {
                kern::add(c, acc.ptr, sums[k].ptr, acc.ptr, 2 * (int)next * nb, ext, (int)next);
            }
        }
        inner.clear();
    }
    for (auto& kv : inner) {
        const int g = kv.first;
        u64* x = kv.second.ptr;
        const long long R = (((long long)p0.a0 + (long long)p0.step * g * p0.B) % m + m) % m;
        if (!R) {
            if (!have_acc) {
                acc = std::move(kv.second);
                have_acc = true;
            } else {
                kern::add(c, acc.ptr, x, acc.ptr, 2 * (int)next * nb, ext, (int)next);
            }
            continue;
        }
        const u64 gal = galois_of_step(c, R);
        c->ops["hrot"]++;
        DevBuf c1q((size_t)nb * nl * n, c->stream);
        mod_down_poly(c, x + next * n, l, c1q.ptr, nb, es);
        int ndig = 0;
        DevBuf D = mod_up(c, c1q.ptr, l, &ndig, nb, (size_t)nl * n);
        if (!have_acc) acc = DevBuf(nb * es, c->stream);
        key_switch_inner(c, keys, D.ptr, ndig, l, gal, gal, acc.ptr, have_acc, x, (int)next, nullptr, nullptr,
                         nullptr, nb, es);
        have_acc = true;
    }
    if (rescale_out) {
        ckks_ct o = new_ct(c, l - 1, scale / (double)c->q[l], nb);
        mod_down_rescale(c, acc.ptr, l, o.buf.ptr, false, nb);
        return o;
    }
    ckks_ct o = new_ct(c, l, scale, nb);
    mod_down(c, acc.ptr, l, o.buf.ptr, nb);
    return o;
}

ckks_ct bsgs(const ckks_keys& keys, const ckks_ct& a, const ckks_ptset& ps, bool rescale_out) {
    return bsgs_multi(keys, {&a}, {&ps}, rescale_out);
}

// ------------------------------------------------ Chebyshev / EvalMod -----
// Ciphertexts of one level and scale gathered into one lockstep batch, and ciphertext t of a batch
// copied out (so that independent products inside one operation share their launches and keys)
static ckks_ct gather_cts(const std::vector<const ckks_ct*>& v) {
    ckks_ctx* c = v[0]->ctx;
    ckks_ct x = new_ct(c, v[0]->level, v[0]->scale, (int)v.size());
    for (size_t t = 0; t < v.size(); ++t) {
        CK_CHECK(v[t]->nb == 1 && v[t]->level == x.level, CKKS_EINVAL, "gathered ciphertexts differ in level");
        CUDA_CHECK(cudaMemcpyAsync(x.c0((int)t), v[t]->buf.ptr, x.cstride() * 8, cudaMemcpyDeviceToDevice, c->stream));
    }
    return x;
}
static ckks_ct take_ct(const ckks_ct& batch, int t) {
    ckks_ctx* c = batch.ctx;
    ckks_ct o = new_ct(c, batch.level, batch.scale);
    CUDA_CHECK(cudaMemcpyAsync(o.buf.ptr, batch.c0(t), batch.cstride() * 8, cudaMemcpyDeviceToDevice, c->stream));
    return o;
}

// Level at which to multiply two ciphertexts available at level m: a product at the
// bottom level of the bootstrapping segment would not rescale onto the circuit segment's
// canonical scale, so it is taken one level lower.
static int prod_level(const ckks_ctx* c, int m) {
    if (c->P.n_boot > 0 && c->n_circuit >= 1 && m == c->n_circuit + 1) return m - 1;
    return m;
}
// level after `depth` multiplicative levels from `level` (one more across the boundary)
static int poly_out_level(const ckks_ctx* c, int level, int depth) {
    int want = level - depth;
    if (c->P.n_boot > 0 && c->n_circuit >= 1 && want <= c->n_circuit && c->n_circuit < level) --want;
    return want;
}

// T_k(x) for the requested k (and what they need): T_k = 2 T_ceil(k/2) T_floor(k/2) -
// T_(k mod 2 ? 1 : 0), operands brought to a common level by level_down.
struct ChebPowers {
    const ckks_keys* keys;
    std::map<int, ckks_ct> T;
    std::map<std::pair<int, int>, ckks_ct> cache;
    const ckks_ct& at(int k, int lev) {
        const ckks_ct& t = T.at(k);
        if (t.level == lev) return t;
        auto key = std::make_pair(k, lev);
        auto it = cache.find(key);
        if (it == cache.end()) it = cache.emplace(key, level_down(t, lev)).first;
        return it->second;
    }
    void need(int k) {
        if (T.count(k)) return;
        const int a = k / 2, b = k - k / 2;
        need(a);
        need(b);
        if (a != b) need(b - a);
        T[k] = product(k);
    }
    // T_k from T_a, T_b (and T_(b-a)), which must exist
    ckks_ct product(int k) {
        const int a = k / 2, b = k - k / 2;
        const int m = prod_level(T.at(a).ctx, std::min(T.at(a).level, T.at(b).level));
        ckks_ct t = mul_relin_rescale(*keys, at(a, m), at(b, m), true);     // 2 T_a T_b
        return (a == b) ? add_const(t, -1.0) : sub(t, at(b - a, m - 1));
    }
    // several T_k at once: the products taken at the same level run as one lockstep batch
    // (one relinearisation key read, every launch over all of them); same residues as product(k)
    void products_batched(const std::vector<int>& ks) {
        std::map<int, std::vector<int>> by_level;
        for (int k : ks) {
            const int a = k / 2, b = k - k / 2;
            by_level[prod_level(T.at(a).ctx, std::min(T.at(a).level, T.at(b).level))].push_back(k);
        }
        for (auto& kv : by_level) {
            const int m = kv.first;
            const std::vector<int>& g = kv.second;
            if (g.size() == 1) {
                T[g[0]] = product(g[0]);
                continue;
            }
            std::vector<const ckks_ct*> xa, xb;
            for (int k : g) {
                xa.push_back(&at(k / 2, m));
                xb.push_back(&at(k - k / 2, m));
            }
            ckks_ct prod = mul_relin_rescale(*keys, gather_cts(xa), gather_cts(xb), true);     // 2 T_a T_b
            for (size_t i = 0; i < g.size(); ++i) {
                const int k = g[i], a = k / 2, b = k - k / 2;
                ckks_ct t = take_ct(prod, (int)i);
                T[k] = (a == b) ? add_const(t, -1.0) : sub(t, at(b - a, m - 1));
            }
        }
    }
    // the level_downs product(k) reads, made ahead (so that products can run side by side)
    void warm(int k) {
        const int a = k / 2, b = k - k / 2;
        const int m = prod_level(T.at(a).ctx, std::min(T.at(a).level, T.at(b).level));
        at(a, m);
        at(b, m);
        if (a != b) at(b - a, m - 1);
    }
};

// Result of evaluating a piece: a ciphertext, or a plain constant when only c_0 is non-zero.
struct PolyVal {
    bool is_const = false;
    double cst = 0.0;
    ckks_ct ct;
};

// sum_k c_k T_k for a piece of degree < b.  The target level is the lowest level among its
// T_k minus one; every T_k is brought to target + 1 by level_down (cached in ChebPowers, so the
// leaves of one polynomial share it), multiplied by llround(c_k s_c), s_c = Delta_target
// q_(target+1) / scale, summed and rescaled once.
static PolyVal cheb_leaf(ChebPowers& pw, const std::vector<double>& c) {
    ckks_ctx* ctx = pw.T.at(1).ctx;
    PolyVal out;
    std::vector<int> ks;
    for (int k = 1; k < (int)c.size(); ++k)
        if (c[k] != 0.0) ks.push_back(k);
    if (ks.empty()) {
        out.is_const = true;
        out.cst = c[0];
        return out;
    }
    int lev = 1 << 30;
    for (int k : ks) lev = std::min(lev, pw.T.at(k).level);
    const int target = lev - 1;
    CK_CHECK((int)ks.size() <= kern::LinComb::MAX, CKKS_EINVAL, "Chebyshev leaf with more than 16 terms");
    kern::LinComb L;
    L.n = 0;
    for (int k : ks) {
        const ckks_ct& t = pw.at(k, lev);
        const double s_c = (ctx->delta[target] * (double)ctx->q[lev]) / t.scale;
        const long long w = llround_away(c[k] * s_c);
        L.a[L.n] = t.buf.ptr;
        for (int i = 0; i <= lev; ++i) {
            L.w[L.n][i] = from_signed(w, ctx->q[i]);
            L.wp[L.n][i] = shoup(L.w[L.n][i], ctx->q[i]);
        }
        ++L.n;
    }
    const int nb = pw.T.at(1).nb;
    ckks_ct acc = new_ct(ctx, lev, 0.0, nb);
    kern::lincomb(ctx, L, acc.buf.ptr, 2 * (lev + 1) * nb, ctx->d_iota, lev + 1);
    acc = rescale(acc);
    acc.scale = ctx->delta[target];
    out.ct = add_const(acc, c[0]);
    return out;
}

// sum_k c_k T_k(x) by baby-step giant-step: baby steps T_1..T_b, giant steps T_b, T_2b, ...
// (b = 2^ceil(m/2), m = ceil(log2(deg + 1))); p = q T_n + r by Chebyshev division (n the
// largest giant <= deg; q_0 = c_n, q_j = 2 c_(n+j), r_(n-j) = c_(n-j) - c_(n+j)) down to
// pieces of degree < b; the result is brought down to level(x) - ceil(log2 deg) - 1.
ckks_ct cheb_eval(const ckks_keys& keys, const ckks_ct& x, const std::vector<double>& coeffs) {
    const int d = (int)coeffs.size() - 1;
    CK_CHECK(d >= 1, CKKS_EINVAL, "polynomial degree must be >= 1");
    int depth = 0;
    while ((1 << depth) < d) ++depth;
    const int want = poly_out_level(x.ctx, x.level, depth + 1);
    CK_CHECK(want >= 0, CKKS_ELEVEL, "not enough levels for the polynomial");
    int m = 0;
    while ((1 << m) < d + 1) ++m;
    const int b = 1 << ((m + 1) / 2);
    std::vector<int> giants;
    for (int n = b; n <= d; n *= 2) giants.push_back(n);
    ChebPowers pw;
    pw.keys = &keys;
    pw.T[1] = copy_ct(x);
    // The leaves (pieces of degree < b) depend only on the baby steps T_1..T_(b-1): collect them
    // in the order the Chebyshev division below visits them.
    auto trim = [](std::vector<double>& c) {
        int deg = (int)c.size() - 1;
        while (deg > 0 && c[deg] == 0.0) --deg;
        c.resize(deg + 1);
    };
    auto split = [&](const std::vector<double>& c, int* n_out, std::vector<double>* q, std::vector<double>* r) {
        const int deg = (int)c.size() - 1;
        int n = 0;
        for (int g : giants)
            if (g <= deg) n = g;
        q->assign(deg - n + 1, 0.0);
        r->assign(c.begin(), c.begin() + n);
        (*q)[0] = c[n];
        for (int j = 1; j <= deg - n; ++j) {
            (*q)[j] = 2.0 * c[n + j];
            (*r)[n - j] -= c[n + j];
        }
        *n_out = n;
    };
    std::vector<std::vector<double>> leaves;
    std::function<void(std::vector<double>)> collect = [&](std::vector<double> c) {
        trim(c);
        if ((int)c.size() - 1 < b) {
            leaves.push_back(c);
            return;
        }
        int n = 0;
        std::vector<double> q, r;
        split(c, &n, &q, &r);
        collect(q);
        collect(r);
    };
    collect(coeffs);
    ckks_ctx* cx = x.ctx;
    // Powers by generations (a generation needs only earlier ones); within a generation the
    // products are independent and, two or more, run on the side streams.  The generations
    // that hold baby steps come first; then the leaves are started on the side streams
    // (every T_k they use brought to its leaf level beforehand, so the shared cache is
    // complete), and the remaining giant steps are built on the context's stream meanwhile.
    std::map<int, int> gen{{1, 0}};
    std::function<int(int)> generation = [&](int k) -> int {
        auto it = gen.find(k);
        if (it != gen.end()) return it->second;
        const int a = k / 2, bb = k - k / 2;
        int g = std::max(generation(a), generation(bb));
        if (a != bb) g = std::max(g, generation(bb - a));
        gen[k] = g + 1;
        return g + 1;
    };
    int baby_gen = 0, maxgen = 0;
    for (int k = 2; k < std::min(b, d + 1); ++k) baby_gen = std::max(baby_gen, generation(k));
    for (int g : giants) generation(g);
    for (const auto& kv : gen) maxgen = std::max(maxgen, kv.second);
    auto fork = [&](int nwork) -> int {
        ensure_side_streams(cx);
        CUDA_CHECK(cudaEventRecord(cx->fork_ev, cx->stream));
        const int nside = std::min(nwork, ckks_ctx::NSIDE);
        for (int k = 0; k < nside; ++k) CUDA_CHECK(cudaStreamWaitEvent(cx->side[k], cx->fork_ev, 0));
        return nside;
    };
    auto join = [&](int nside, cudaStream_t main_stream) {
        for (int k = 0; k < nside; ++k) {
            CUDA_CHECK(cudaEventRecord(cx->side_ev[k], cx->side[k]));
            CUDA_CHECK(cudaStreamWaitEvent(main_stream, cx->side_ev[k], 0));
        }
    };
    auto run_generations = [&](int g0, int g1) {
        for (int g = g0; g <= g1; ++g) {
            std::vector<int> ks;
            for (const auto& kv : gen)
                if (kv.second == g && !pw.T.count(kv.first)) ks.push_back(kv.first);
            if (ks.empty()) continue;
            for (int k : ks) pw.warm(k);
            if (cx->inner_batching && ks.size() >= 2) {
                pw.products_batched(ks);
                continue;
            }
            if (!cx->use_side_streams() || ks.size() < 2) {
                for (int k : ks) pw.T[k] = pw.product(k);
                continue;
            }
            const cudaStream_t main_stream = cx->stream;
            StreamRestore restore{cx, main_stream};
            const int nside = fork((int)ks.size());
            for (size_t i = 0; i < ks.size(); ++i) {
                cx->stream = cx->side[i % ckks_ctx::NSIDE];
                pw.T[ks[i]] = pw.product(ks[i]);
            }
            join(nside, main_stream);
            cx->stream = main_stream;
            for (int k : ks) pw.T[k].buf.stream = main_stream;
        }
    };
    run_generations(1, baby_gen);
    for (const auto& c : leaves) {
        int lev = 1 << 30;
        for (int k = 1; k < (int)c.size(); ++k)
            if (c[k] != 0.0) lev = std::min(lev, pw.T.at(k).level);
        for (int k = 1; k < (int)c.size(); ++k)
            if (c[k] != 0.0) pw.at(k, lev);
    }
    std::vector<PolyVal> leaf_vals(leaves.size());
    if (cx->use_side_streams() && leaves.size() >= 2) {
        const cudaStream_t main_stream = cx->stream;
        int nside = 0;
        {
            StreamRestore restore{cx, main_stream};
            nside = fork((int)leaves.size());
            for (size_t i = 0; i < leaves.size(); ++i) {
                cx->stream = cx->side[i % ckks_ctx::NSIDE];
                leaf_vals[i] = cheb_leaf(pw, leaves[i]);
            }
        }
        run_generations(baby_gen + 1, maxgen);       // on the context's stream, beside the leaves
        join(nside, main_stream);
        for (auto& v : leaf_vals)       // freed later on the context's stream, after its uses there
            if (!v.is_const) v.ct.buf.stream = main_stream;
    } else {
        for (size_t i = 0; i < leaves.size(); ++i) leaf_vals[i] = cheb_leaf(pw, leaves[i]);
        run_generations(baby_gen + 1, maxgen);
    }
    // The division as a tree (children visited Q before R, leaves in the same order as above);
    // internal nodes are combined by height: nodes of one height are independent and, two or
    // more, run on the side streams (the level_downs of T_n they read are made first).
    struct Node {
        int n = 0, q = -1, r = -1, leaf = -1, height = 0;
        PolyVal val;
    };
    std::vector<Node> nodes;
    int leaf_counter = 0;
    std::function<int(std::vector<double>)> build = [&](std::vector<double> c) -> int {
        trim(c);
        const int id = (int)nodes.size();
        nodes.emplace_back();
        if ((int)c.size() - 1 < b) {
            nodes[id].leaf = leaf_counter++;
            return id;
        }
        int n = 0;
        std::vector<double> q, r;
        split(c, &n, &q, &r);
        const int qi = build(q);
        const int ri = build(r);
        nodes[id].n = n;
        nodes[id].q = qi;
        nodes[id].r = ri;
        nodes[id].height = 1 + std::max(nodes[qi].height, nodes[ri].height);
        return id;
    };
    const int root = build(coeffs);
    for (auto& nd : nodes)
        if (nd.leaf >= 0) nd.val = std::move(leaf_vals[nd.leaf]);
    auto prod_lev = [&](const Node& nd) {
        const ckks_ct& Tn = pw.T.at(nd.n);
        return prod_level(Tn.ctx, std::min(nodes[nd.q].val.ct.level, Tn.level));
    };
    auto combine = [&](Node& nd) -> PolyVal {
        PolyVal& Q = nodes[nd.q].val;
        PolyVal& R = nodes[nd.r].val;
        const ckks_ct& Tn = pw.T.at(nd.n);
        ckks_ctx* ctx = Tn.ctx;
        ckks_ct prod;
        bool hp = false;
        if (Q.is_const) {
            if (Q.cst != 0.0) {
                const int lk = Tn.level;
                const double s_c = (ctx->delta[lk - 1] * (double)ctx->q[lk]) / Tn.scale;
                prod = rescale_mul(Tn, llround_away(Q.cst * s_c));
                prod.scale = (Tn.scale * s_c) / (double)ctx->q[lk];
                hp = true;
            }
        } else {
            const int lev = prod_lev(nd);
            prod = mul_relin_rescale(keys, level_down(Q.ct, lev), pw.at(nd.n, lev));
            hp = true;
        }
        PolyVal out;
        if (R.is_const) {
            if (!hp) return std::move(R);
            out.ct = add_const(prod, R.cst);
            return out;
        }
        if (!hp) return std::move(R);
        const int lev = std::min(prod.level, R.ct.level);
        out.ct = add(level_down(prod, lev), level_down(R.ct, lev));
        return out;
    };
    for (int h = 1; h <= nodes[root].height; ++h) {
        std::vector<int> ids;
        for (int i = 0; i < (int)nodes.size(); ++i)
            if (nodes[i].leaf < 0 && nodes[i].height == h) ids.push_back(i);
        for (int i : ids)
            if (!nodes[nodes[i].q].val.is_const) pw.at(nodes[i].n, prod_lev(nodes[i]));
        if (!cx->use_side_streams() || ids.size() < 2) {
            for (int i : ids) nodes[i].val = combine(nodes[i]);
        } else {
            ensure_side_streams(cx);
            const cudaStream_t main_stream = cx->stream;
            StreamRestore restore{cx, main_stream};
            CUDA_CHECK(cudaEventRecord(cx->fork_ev, main_stream));
            const int nside = std::min((int)ids.size(), ckks_ctx::NSIDE);
            for (int k = 0; k < nside; ++k) CUDA_CHECK(cudaStreamWaitEvent(cx->side[k], cx->fork_ev, 0));
            for (size_t k = 0; k < ids.size(); ++k) {
                cx->stream = cx->side[k % ckks_ctx::NSIDE];
                nodes[ids[k]].val = combine(nodes[ids[k]]);
            }
            for (int k = 0; k < nside; ++k) {
                CUDA_CHECK(cudaEventRecord(cx->side_ev[k], cx->side[k]));
                CUDA_CHECK(cudaStreamWaitEvent(main_stream, cx->side_ev[k], 0));
            }
            cx->stream = main_stream;
            for (int i : ids)
                if (!nodes[i].val.is_const) nodes[i].val.ct.buf.stream = main_stream;
        }
        for (int i : ids) {          // the children are consumed (after the join)
            nodes[nodes[i].q].val = PolyVal();
            nodes[nodes[i].r].val = PolyVal();
        }
    }
    PolyVal res = std::move(nodes[root].val);
    CK_CHECK(!res.is_const, CKKS_EINVAL, "polynomial evaluates to a constant");
    CK_CHECK(res.ct.level >= want, CKKS_ELEVEL, "polynomial evaluation ended below its level budget");
    return level_down(res.ct, want);
}

// HActivation as a composite polynomial: y = s_k(...s_1(x)) by chained Chebyshev
// evaluations, then x y with x brought down to y's level
ckks_ct eval_relu(const ckks_keys& keys, const ckks_ct& x, const std::vector<std::vector<double>>& stages) {
    CK_CHECK(!stages.empty(), CKKS_EINVAL, "no activation stages");
    ckks_ct y = cheb_eval(keys, x, stages[0]);
    for (size_t i = 1; i < stages.size(); ++i) y = cheb_eval(keys, y, stages[i]);
    const int lev = prod_level(x.ctx, y.level);
    CK_CHECK(lev >= 1, CKKS_ELEVEL, "not enough levels for the final product");
    return mul_relin_rescale(keys, level_down(x, lev), level_down(y, lev));
}

// alpha x + beta: x times llround(alpha Delta_(l-1) q_l / scale), rescaled onto the canonical
// scale Delta_(l-1) (one level), then beta added
ckks_ct affine(const ckks_ct& x, double alpha, double beta) {
    ckks_ctx* c = x.ctx;
    const int l = x.level;
    CK_CHECK(l >= 1, CKKS_ELEVEL, "not enough levels for the change of variable");
    ckks_ct y = rescale_mul(x, llround_away(alpha * (c->delta[l - 1] * (double)c->q[l]) / x.scale));
    y.scale = c->delta[l - 1];
    return add_const(y, beta);
}

// p(x) on [a, b]: y = (2x - a - b) / (b - a) (no level for [-1, 1]), a power-basis p re-expressed
// as a Chebyshev series in y on the host, then cheb_eval
ckks_ct eval_poly(const ckks_keys& keys, const ckks_ct& x, const std::vector<double>& coeffs, bool power, double a,
                  double b) {
    CK_CHECK(b > a, CKKS_EINVAL, "the interval needs a < b");
    const double alpha = 2.0 / (b - a), beta = -(a + b) / (b - a);
    std::vector<double> ch = power ? fp64::power_to_cheb(coeffs, alpha, beta) : coeffs;
    if (a == -1.0 && b == 1.0) return cheb_eval(keys, x, ch);
    return cheb_eval(keys, affine(x, alpha, beta), ch);
}

ckks_ct eval_mod(const ckks_keys& keys, const ckks_ct& x, const std::vector<double>& coeffs, int r) {
    ckks_ct y = cheb_eval(keys, x, coeffs);
    for (int i = 0; i < r; ++i) {
        y = mul_relin_rescale(keys, y, y, true);     // 2 y^2
        y = add_const(y, -1.0);
    }
    return y;
}

void bootstrap(const ckks_keys& keys, const ckks_boot& bt, const ckks_ct& ct0, ckks_ct& re_out, ckks_ct& im_out) {
    ckks_ctx* c = ct0.ctx;
    ckks_ct x = mod_raise(ct0);
    x.scale = bt.s_raise;
    for (const auto& ps : bt.ctos) x = bsgs(keys, x, *ps, true);
    ckks_ct cj = conjugate(keys, x);
    ckks_ct re = add(x, cj);
    ckks_ct im = imult(sub(cj, x));
    re = rescale_mul(re, bt.c_drop);
    im = rescale_mul(im, bt.c_drop);
    re.scale = c->delta[re.level];
    im.scale = c->delta[im.level];
    re_out = eval_mod(keys, re, bt.coeffs, bt.bp.r);
    im_out = eval_mod(keys, im, bt.coeffs, bt.bp.r);
}

// recombined slot ciphertext -> [Alg. 2 decomposition] -> HMatmul(S_{l'<-1})
static ckks_ct tail(const ckks_keys& keys, const ckks_boot& bt, ckks_ct y) {
    if (bt.decomp) y = bsgs(keys, y, *bt.decomp, true);
    for (const auto& ps : bt.stoc) y = bsgs(keys, y, *ps, true);
    return y;
}

static ckks_ct boot_tail(const ckks_keys& keys, const ckks_boot& bt, const ckks_ct& x0);

// Alg. 1 block.  When the Im mask is exactly zero (the second half of every slice is
// padding), PMult(ct_Im, mask_Im) is the zero ciphertext whatever ct_Im holds, so the Im
// branch (its scale drop and EvalMod) is skipped; the output is bit-identical.
ckks_ct block(const ckks_keys& keys, const ckks_boot& bt, const ckks_ptset& conv, const ckks_ct& in) {
    return boot_tail(keys, bt, bsgs(keys, in, conv, true));
}

// conv over several input ciphertexts (BSGS each, HAdd, one rescale), then the block's
// bootstrap and tail: with the decomposed stride-2 kernels, Alg. 2 from the decomposed convs
// to the end; otherwise the C_in > C block matrix-vector product (Sec. 3.3.3).
ckks_ct block_multi(const ckks_keys& keys, const ckks_boot& bt, const std::vector<const ckks_ptset*>& convs,
                    const std::vector<const ckks_ct*>& ins) {
    return boot_tail(keys, bt, bsgs_multi(keys, ins, convs, true));
}

// Alg. 2 without HActivation: per input, the stride-2 tail of the previous block (masks,
// Re + i Im, decomposition, S_{l/4<-1}) and a level drop to the conv's level; then the
// decomposed convs, one bootstrap and the tail of bt_out.
ckks_ct downsample_layer(const ckks_keys& keys, const ckks_boot& bt_in, const ckks_boot& bt_out,
                         const std::vector<const ckks_ct*>& re, const std::vector<const ckks_ct*>& im,
                         const std::vector<const ckks_ptset*>& convs) {
    std::vector<ckks_ct> ys;
    ys.reserve(re.size());
    for (size_t t = 0; t < re.size(); ++t) ys.push_back(level_down(stoc1(keys, bt_in, *re[t], *im[t]), convs[t]->level));
    std::vector<const ckks_ct*> ptrs;
    for (const ckks_ct& y : ys) ptrs.push_back(&y);
    return block_multi(keys, bt_out, convs, ptrs);
}

static ckks_ct boot_tail(const ckks_keys& keys, const ckks_boot& bt, const ckks_ct& x0) {
    ckks_ctx* c = x0.ctx;
    if (!bt.mask_im_zero) {
        ckks_ct re, im;
        bootstrap(keys, bt, x0, re, im);
        return stoc1(keys, bt, re, im);
    }
    ckks_ct x = mod_raise(x0);
    x.scale = bt.s_raise;
    for (const auto& ps : bt.ctos) x = bsgs(keys, x, *ps, true);
    ckks_ct re = add(x, conjugate(keys, x));
    re = rescale_mul(re, bt.c_drop);
    re.scale = c->delta[re.level];
    re = eval_mod(keys, re, bt.coeffs, bt.bp.r);
    return tail(keys, bt, rescale(mul_plain(re, *bt.mask_re)));
}

ckks_ct stoc1(const ckks_keys& keys, const ckks_boot& bt, const ckks_ct& re, const ckks_ct& im) {
    ckks_ct a = rescale(mul_plain(re, *bt.mask_re));
    ckks_ct b = rescale(mul_plain(im, *bt.mask_im));
    return tail(keys, bt, add(a, imult(b)));
}

}  // namespace ops

// ================================================================ keys =====
namespace ops {

static void gen_switch_key(ckks_ctx* c, ckks_keys& K, u64 code, const u64* sprime_ntt) {
    const size_t n = c->n;
    std::vector<std::vector<int>> dig = c->digits(c->L);
    auto sk = std::make_unique<SwitchKey>();
    sk->ndig = (int)dig.size();
    const size_t per = (size_t)c->nall * n;
    sk->b = DevBuf(sk->ndig * per, c->stream);
    sk->a = DevBuf(sk->ndig * per, c->stream);
    DevBuf e_small(n, c->stream);
    std::vector<u64> pm(2 * c->nq);
    for (int i = 0; i < c->nq; ++i) {
        u64 v = 1;
        for (u64 pj : c->p) v = mulmod(v, pj % c->q[i], c->q[i]);
        pm[i] = v;
        pm[c->nq + i] = shoup(v, c->q[i]);
    }
    DevBuf dpm = upload(c, pm);
    DevBuf tmp(n, c->stream);
    for (int d = 0; d < sk->ndig; ++d) {
        u64* a = sk->a.ptr + d * per;
        u64* b = sk->b.ptr + d * per;
        kern::sample_uniform(c, a, c->nall, c->d_iota, stream_key(c->seed, tag(K_SWK_A, code, d)));
        kern::sample_small(c, (int64_t*)e_small.ptr, stream_key(c->seed, tag(K_SWK_E, code, d)), 1);
        kern::small_to_rns(c, (const int64_t*)e_small.ptr, b, c->nall, c->d_iota);
        kern::ntt_forward(c, b, c->nall, c->d_iota, c->nall);
        DevBuf as(per, c->stream);
        kern::mul(c, a, K.s_ntt.ptr, as.ptr, c->nall, c->d_iota, c->nall);
        kern::sub(c, b, as.ptr, b, c->nall, c->d_iota, c->nall);
        for (int i : dig[d]) {
            kern::mul_scalar(c, sprime_ntt + (size_t)i * n, dpm.ptr + i, dpm.ptr + c->nq + i, tmp.ptr, 1,
                             c->d_iota + i, 1);
            kern::add(c, b + (size_t)i * n, tmp.ptr, b + (size_t)i * n, 1, c->d_iota + i, 1);
        }
    }
    K.swk[code] = std::move(sk);
}

void add_galois_key(ckks_ctx* c, ckks_keys& K, u64 g) {
    if (g == 1 || K.swk.count(g)) return;
    DevBuf sg((size_t)c->nall * c->n, c->stream);
    kern::automorph(c, K.s_ntt.ptr, sg.ptr, c->nall, g);
    gen_switch_key(c, K, g, sg.ptr);
}

ckks_keys* keygen(ckks_ctx* c, const int32_t* steps, int nsteps, int want_conj) {
    const size_t n = c->n;
    std::unique_ptr<ckks_keys> K(new ckks_keys());
    K->ctx = c;
    K->s.assign(n, 0);
    if (c->P.h > 0) {
        CK_CHECK(c->P.h <= c->n, CKKS_EINVAL, "Hamming weight above N");
        u64 kp = stream_key(c->seed, tag(K_SK)), ks = stream_key(c->seed, tag(K_SK_SIGN));
        std::vector<int> perm(n);
        for (size_t j = 0; j < n; ++j) perm[j] = (int)j;
        for (int i = 0; i < c->P.h; ++i) {
            int r = (int)(stream_word(kp, i) % (u64)(n - i));
            std::swap(perm[i], perm[i + r]);
            K->s[perm[i]] = (stream_word(ks, i) & 1) ? -1 : 1;
        }
    } else {
        u64 key = stream_key(c->seed, tag(K_SK));
        for (size_t j = 0; j < n; ++j) K->s[j] = (int64_t)(stream_word(key, j) % 3) - 1;
    }
    DevBuf s_small(n, c->stream);
    CUDA_CHECK(cudaMemcpyAsync(s_small.ptr, K->s.data(), n * 8, cudaMemcpyHostToDevice, c->stream));
    K->s_ntt = DevBuf((size_t)c->nall * n, c->stream);
    kern::small_to_rns(c, (const int64_t*)s_small.ptr, K->s_ntt.ptr, c->nall, c->d_iota);
    kern::ntt_forward(c, K->s_ntt.ptr, c->nall, c->d_iota, c->nall);
    // public key over Q_L
    const int nq = c->nq;
    K->pk_a = DevBuf((size_t)nq * n, c->stream);
    K->pk_b = DevBuf((size_t)nq * n, c->stream);
    kern::sample_uniform(c, K->pk_a.ptr, nq, c->d_iota, stream_key(c->seed, tag(K_PK_A)));
    DevBuf e(n, c->stream);
    kern::sample_small(c, (int64_t*)e.ptr, stream_key(c->seed, tag(K_PK_E)), 1);
    kern::small_to_rns(c, (const int64_t*)e.ptr, K->pk_b.ptr, nq, c->d_iota);
    kern::ntt_forward(c, K->pk_b.ptr, nq, c->d_iota, nq);
    DevBuf as((size_t)nq * n, c->stream);
    kern::mul(c, K->pk_a.ptr, K->s_ntt.ptr, as.ptr, nq, c->d_iota, nq);
    kern::sub(c, K->pk_b.ptr, as.ptr, K->pk_b.ptr, nq, c->d_iota, nq);
    // relinearisation key: s' = s^2
    DevBuf s2((size_t)c->nall * n, c->stream);
    kern::mul(c, K->s_ntt.ptr, K->s_ntt.ptr, s2.ptr, c->nall, c->d_iota, c->nall);
    gen_switch_key(c, *K, 0, s2.ptr);
    for (int i = 0; i < nsteps; ++i) add_galois_key(c, *K, galois_of_step(c, steps[i]));
    if (want_conj) add_galois_key(c, *K, 2ULL * c->n - 1);
    return K.release();
}

// ========================================================== encryption =====
ckks_ct encrypt(const ckks_keys& K, const ckks_pt& pt, u64 nonce) {
    ckks_ctx* c = K.ctx;
    const int l = pt.level, nl = l + 1;
    const size_t n = c->n;
    ckks_ct o = new_ct(c, l, pt.scale);
    DevBuf sm(n, c->stream), u(nl * n, c->stream), e(nl * n, c->stream);
    kern::sample_small(c, (int64_t*)sm.ptr, stream_key(c->seed, tag(K_ENC_U, nonce)), 0);
    kern::small_to_rns(c, (const int64_t*)sm.ptr, u.ptr, nl, c->d_iota);
    kern::ntt_forward(c, u.ptr, nl, c->d_iota, nl);
    // c0 = u b + e0 + m
    kern::sample_small(c, (int64_t*)sm.ptr, stream_key(c->seed, tag(K_ENC_E0, nonce)), 1);
    kern::small_to_rns(c, (const int64_t*)sm.ptr, e.ptr, nl, c->d_iota);
    kern::ntt_forward(c, e.ptr, nl, c->d_iota, nl);
    kern::add(c, e.ptr, pt.buf.ptr, o.c0(), nl, c->d_iota, nl);
    kern::mul_acc(c, u.ptr, K.pk_b.ptr, o.c0(), nl, c->d_iota, nl);
    // c1 = u a + e1
    kern::sample_small(c, (int64_t*)sm.ptr, stream_key(c->seed, tag(K_ENC_E1, nonce)), 1);
    kern::small_to_rns(c, (const int64_t*)sm.ptr, o.c1(), nl, c->d_iota);
    kern::ntt_forward(c, o.c1(), nl, c->d_iota, nl);
    kern::mul_acc(c, u.ptr, K.pk_a.ptr, o.c1(), nl, c->d_iota, nl);
    return o;
}

ckks_ct encrypt_sk(const ckks_keys& K, const ckks_pt& pt, u64 nonce) {
    ckks_ctx* c = K.ctx;
    const int l = pt.level, nl = l + 1;
    const size_t n = c->n;
    ckks_ct o = new_ct(c, l, pt.scale);
    DevBuf sm(n, c->stream), as(nl * n, c->stream);
    kern::sample_uniform(c, o.c1(), nl, c->d_iota, stream_key(c->seed, tag(K_ENCSK_A, nonce)));
    kern::sample_small(c, (int64_t*)sm.ptr, stream_key(c->seed, tag(K_ENCSK_E, nonce)), 1);
    kern::small_to_rns(c, (const int64_t*)sm.ptr, o.c0(), nl, c->d_iota);
    kern::ntt_forward(c, o.c0(), nl, c->d_iota, nl);
    kern::mul(c, o.c1(), K.s_ntt.ptr, as.ptr, nl, c->d_iota, nl);
    kern::sub(c, o.c0(), as.ptr, o.c0(), nl, c->d_iota, nl);
    kern::add(c, o.c0(), pt.buf.ptr, o.c0(), nl, c->d_iota, nl);
    return o;
}

void decrypt(const ckks_keys& K, const ckks_ct& ct, ckks_pt& out) {
    ckks_ctx* c = K.ctx;
    CK_CHECK(ct.nb == 1, CKKS_EINVAL, "decrypt takes a single ciphertext");
    const int nl = ct.level + 1;
    DevBuf m((size_t)nl * c->n, c->stream);
    kern::mul(c, ct.c1(), K.s_ntt.ptr, m.ptr, nl, c->d_iota, nl);
    kern::add(c, m.ptr, ct.c0(), m.ptr, nl, c->d_iota, nl);
    out.ctx = c;
    out.buf = std::move(m);
    out.level = ct.level;
    out.scale = ct.scale;
}

}  // namespace ops
