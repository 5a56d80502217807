// extern "C" entry points (include/ckks.h).  Each call catches every C++ error and
// returns a status code; ckks_last_error(ctx) keeps the message.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <set>

#include "internal.h"
#include "scheme_ops.h"

using namespace hostmath;

namespace {

// Puts the calling context's allocator in place for the call (DevBufs made during it take
// their memory from it) and restores the previous one afterwards, also on an exception.
struct AllocScope {
    const DevAlloc* prev;
    explicit AllocScope(const ckks_ctx* c) : prev(tl_alloc) { tl_alloc = c && c->alloc.alloc ? &c->alloc : nullptr; }
    ~AllocScope() { tl_alloc = prev; }
};

template <class F>
int guard(const ckks_ctx* c, F&& f) {
    try {
        AllocScope scope(c);
        f();
        return CKKS_OK;
    } catch (const CkksError& e) {
        if (c) const_cast<ckks_ctx*>(c)->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (c) const_cast<ckks_ctx*>(c)->err = "host allocation failed";
        return CKKS_ENOMEM;
    } catch (const std::exception& e) {
        if (c) const_cast<ckks_ctx*>(c)->err = e.what();
        return CKKS_EINVAL;
    }
}

#define REQ(p) CK_CHECK((p) != nullptr, CKKS_EINVAL, #p " is NULL")
#define CT_OK(x) CK_CHECK((x) && (x)->level >= 0, CKKS_EINVAL, #x " is NULL or empty")

void upload_coeffs(ckks_ctx* c, const std::vector<int64_t>& v, int level, double scale, ckks_pt* out,
                   bool ext = false) {
    const size_t n = c->n;
    const int rows = level + 1 + (ext ? c->np : 0);
    const int* ids = ext ? c->d_ext_ids[level] : c->d_iota;
    DevBuf sm(n, c->stream);
    CUDA_CHECK(cudaMemcpyAsync(sm.ptr, v.data(), n * 8, cudaMemcpyHostToDevice, c->stream));
    out->ctx = c;
    out->buf = DevBuf((size_t)rows * n, c->stream);
    out->level = level;
    out->scale = scale;
    out->ext = ext;
    kern::small_to_rns(c, (const int64_t*)sm.ptr, out->buf.ptr, rows, ids);
    kern::ntt_forward(c, out->buf.ptr, rows, ids, rows);
}

std::vector<int64_t> round_coeffs(const std::vector<double>& f, double scale) {
    std::vector<int64_t> v(f.size());
    for (size_t k = 0; k < f.size(); ++k) {
        double x = f[k] * scale;
        CK_CHECK(fabs(x) < ldexp(1.0, 62), CKKS_EINVAL, "encoded coefficient exceeds 2^62");
        v[k] = llround_away(x);
    }
    return v;
}

void encode_complex(ckks_ctx* c, const std::vector<cplx>& z, int level, double scale, ckks_pt* out,
                    bool ext = false) {
    CK_CHECK(level >= 0 && level <= c->L, CKKS_EINVAL, "level out of range");
    std::vector<cplx> zz(z);
    zz.resize(c->n / 2, cplx(0, 0));
    upload_coeffs(c, round_coeffs(fp64::encode_slots(zz, c->n), scale), level, scale, out, ext);
}

// limbs (host, coefficient domain, [nl][N]) -> centred values / scale, by Garner's mixed radix
std::vector<double> crt_centred(const ckks_ctx* c, const std::vector<u64>& limbs, int nl) {
    const size_t n = c->n;
    std::vector<double> out(n);
    // inverse of prod_{k<i} q_k mod q_i
    std::vector<u64> pinv(nl);
    for (int i = 0; i < nl; ++i) {
        u64 pr = 1;
        for (int k = 0; k < i; ++k) pr = mulmod(pr, c->q[k] % c->q[i], c->q[i]);
        pinv[i] = i ? invmod(pr, c->q[i]) : 1;
    }
    std::vector<u64> v(nl);
    for (size_t j = 0; j < n; ++j) {
        bool neg = false;
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = 0; i < nl; ++i) {
                u64 qi = c->q[i];
                u64 r = limbs[(size_t)i * n + j];
                if (neg) r = r ? qi - r : 0;
                // v_i = (r - sum_{t<i} v_t prod_{k<t} q_k) * (prod_{k<i} q_k)^{-1} mod q_i
                u64 acc = 0, pr = 1;
                for (int t = 0; t < i; ++t) {
                    acc = (acc + mulmod(v[t] % qi, pr, qi)) % qi;
                    pr = mulmod(pr, c->q[t] % qi, qi);
                }
                u64 diff = r >= acc ? r - acc : r + qi - acc;
                v[i] = mulmod(diff, pinv[i], qi);
            }
            if (pass == 0 && v[nl - 1] > (c->q[nl - 1] - 1) / 2) {
                neg = true;
                continue;
            }
            break;
        }
        double x = 0.0;
        for (int i = nl - 1; i >= 0; --i) x = x * (double)c->q[i] + (double)v[i];
        out[j] = neg ? -x : x;
    }
    return out;
}

std::vector<u64> download(ckks_ctx* c, const u64* dev, size_t words) {
    std::vector<u64> h(words);
    CUDA_CHECK(cudaMemcpyAsync(h.data(), dev, words * 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
    return h;
}

ckks_ptset* make_plan(ckks_ctx* c, const fp64::Diag& D, int a0, int step, int count, int level, double scale,
                      int B) {
    const int m = c->n / 2;
    std::unique_ptr<ckks_ptset> ps(new ckks_ptset());
    ps->ctx = c;
    ps->a0 = ((a0 % m) + m) % m;
    ps->step = step;
    ps->count = count;
    ps->B = B > 0 ? B : fp64::default_bsgs_B(count);
    ps->level = level;
    ps->scale = scale;
    for (int g = 0; g < ps->G(); ++g) {
        const long long R = ((long long)ps->a0 + (long long)step * g * ps->B) % m;
        for (int b = 0; b < ps->B; ++b) {
            const int i = g * ps->B + b;
            if (i >= count) break;
            const int off = (int)(((long long)ps->a0 + (long long)step * i) % m);
            auto it = D.find(off);
            if (it == D.end()) continue;
            std::vector<cplx> v(m);
            for (int t = 0; t < m; ++t) v[t] = it->second[((t - R) % m + m) % m];
            auto pt = std::make_unique<ckks_pt>();
            encode_complex(c, v, level, scale, pt.get(), true);     // over Q_level u P (double hoisting)
            ps->pts[std::make_pair(g, b)] = std::move(pt);
        }
    }
    return ps.release();
}

void assign(ckks_ct* out, ckks_ct&& v) {
    ckks_ctx* c = v.ctx;
    *out = std::move(v);
    out->ctx = c;
}

}  // namespace

extern "C" {

// ------------------------------------------------------------- context ------
int ckks_ctx_create(const ckks_params* params, uint64_t seed, void* stream, ckks_ctx** out) {
    if (!params || !out) return CKKS_EINVAL;
    try {
        *out = ctx_create(params, seed, (cudaStream_t)stream);
        return CKKS_OK;
    } catch (const CkksError& e) {
        fprintf(stderr, "ckks_ctx_create: %s\n", e.msg.c_str());
        return e.code;
    } catch (...) {
        return CKKS_EINVAL;
    }
}

int ckks_ctx_destroy(ckks_ctx* ctx) {
    delete ctx;
    return CKKS_OK;
}

const char* ckks_last_error(const ckks_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int ckks_sync(ckks_ctx* ctx) {
    return guard(ctx, [&] {
        REQ(ctx);
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        CUDA_CHECK(cudaGetLastError());
        CK_CHECK(kern::peek_device_faults() == 0, CKKS_ETIMEOUT,
                 "a bounded device wait gave up (ckks_ctx_take_device_faults reads and clears the count)");
    });
}

int ckks_ctx_info(const ckks_ctx* ctx, uint64_t* q, uint64_t* p, uint64_t* psi, double* delta) {
    return guard(ctx, [&] {
        REQ(ctx);
        if (q) std::copy(ctx->q.begin(), ctx->q.end(), q);
        if (p) std::copy(ctx->p.begin(), ctx->p.end(), p);
        if (psi) std::copy(ctx->psi.begin(), ctx->psi.end(), psi);
        if (delta) std::copy(ctx->delta.begin(), ctx->delta.end(), delta);
    });
}

int ckks_ctx_gauss_table(const ckks_ctx* ctx, uint64_t* t) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(t);
        std::copy(ctx->gauss, ctx->gauss + 39, t);
    });
}

// ---------------------------------------------------------- measurement -----
int ckks_ctx_set_timing(ckks_ctx* ctx, int on) {
    return guard(ctx, [&] {
        REQ(ctx);
        if (!on) ctx->collect_timing();
        ctx->timing = on != 0;
    });
}

int ckks_ctx_set_pdl(ckks_ctx* ctx, int on) {
    return guard(ctx, [&] {
        REQ(ctx);
        ctx->pdl = on != 0;
    });
}

int ckks_ctx_set_allocator(ckks_ctx* ctx, ckks_alloc_fn alloc, ckks_free_fn free_fn, void* user) {
    return guard(ctx, [&] {
        REQ(ctx);
        CK_CHECK((alloc == nullptr) == (free_fn == nullptr), CKKS_EINVAL, "give both alloc and free_fn, or neither");
        ctx->alloc.alloc = alloc;
        ctx->alloc.free = free_fn;
        ctx->alloc.user = alloc ? user : nullptr;
    });
}

int ckks_ctx_pool_stats(ckks_ctx* ctx, int reset_high, uint64_t* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(out);
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        int dev = 0;
        CUDA_CHECK(cudaGetDevice(&dev));
        cudaMemPool_t pool;
        CUDA_CHECK(cudaDeviceGetDefaultMemPool(&pool, dev));
        if (reset_high) {
            uint64_t zero = 0;
            CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
            CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReservedMemHigh, &zero));
        }
        const cudaMemPoolAttr attrs[4] = {cudaMemPoolAttrUsedMemCurrent, cudaMemPoolAttrUsedMemHigh,
                                          cudaMemPoolAttrReservedMemCurrent, cudaMemPoolAttrReservedMemHigh};
        for (int k = 0; k < 4; ++k) {
            uint64_t v = 0;
            CUDA_CHECK(cudaMemPoolGetAttribute(pool, attrs[k], &v));
            out[k] = v;
        }
    });
}

int ckks_ctx_set_inner_batching(ckks_ctx* ctx, int on) {
    return guard(ctx, [&] {
        REQ(ctx);
        ctx->inner_batching = on != 0;
    });
}

int ckks_ctx_set_tensor_conversion(ckks_ctx* ctx, int mode) {
    return guard(ctx, [&] {
        REQ(ctx);
        CK_CHECK(mode >= 0 && mode <= 2, CKKS_EINVAL, "tensor conversion mode must be 0, 1 or 2");
        ctx->conv_tc = mode != 0;
        if (mode) ctx->conv_tc_tpr = mode;
    });
}

int ckks_debug_withhold_tensor_commit(ckks_ctx* ctx, int on) {
    return guard(ctx, [&] {
        REQ(ctx);
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        kern::set_tc_withhold(on != 0);
    });
}

int ckks_ctx_take_device_faults(ckks_ctx* ctx, uint32_t* count) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(count);
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        *count = kern::take_device_faults();
    });
}

int ckks_ctx_set_side_streams(ckks_ctx* ctx, int on) {
    return guard(ctx, [&] {
        REQ(ctx);
        ctx->side_streams_on = on != 0;
    });
}

int ckks_ctx_counters(const ckks_ctx* ctx, int64_t* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(out);
        auto get = [&](const char* k) {
            auto it = ctx->ops.find(k);
            return it == ctx->ops.end() ? 0L : it->second;
        };
        out[0] = ctx->launches;
        out[1] = get("keyswitch");
        out[2] = get("pmult");
        out[3] = get("hrot");
        out[4] = get("hmult");
        out[5] = get("rescale");
    });
}

int ckks_ctx_reset_counters(ckks_ctx* ctx) {
    return guard(ctx, [&] {
        REQ(ctx);
        ctx->collect_timing();
        ctx->ops.clear();
        ctx->launches = 0;
        ctx->kstats.clear();
    });
}

int ckks_ctx_kernel_stats(ckks_ctx* ctx, char* buf, int cap, int* len) {
    return guard(ctx, [&] {
        REQ(ctx);
        ctx->collect_timing();
        std::string js = "{";
        bool first = true;
        for (const auto& kv : ctx->kstats) {
            char tmp[256];
            snprintf(tmp, sizeof(tmp), "%s\"%s\": [%lld, %.6f, %.1f]", first ? "" : ", ", kv.first.c_str(),
                     kv.second.launches, kv.second.ms, kv.second.bytes);
            js += tmp;
            first = false;
        }
        js += "}";
        if (len) *len = (int)js.size();
        if (buf && cap > 0) {
            int k = std::min((int)js.size(), cap - 1);
            memcpy(buf, js.data(), k);
            buf[k] = 0;
        }
    });
}

int ckks_autotune(ckks_ctx* ctx, int reps, int32_t* choice8) {
    return guard(ctx, [&] {
        REQ(ctx);
        kern::autotune_ntt(ctx, reps > 0 ? reps : 3);
        if (choice8)
            for (int i = 0; i < 8; ++i) choice8[i] = ctx->ntt_choice[i];
    });
}

int ckks_ctx_set_ntt_variant(ckks_ctx* ctx, int variant) {
    return guard(ctx, [&] {
        REQ(ctx);
        CK_CHECK(variant >= -1 && variant <= 5, CKKS_EINVAL, "variant must be -1..5");
        for (int i = 0; i < 8; ++i) ctx->ntt_choice[i] = variant;
    });
}

int ckks_ctx_set_ntt_choices(ckks_ctx* ctx, const int32_t* choice8) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(choice8);
        for (int i = 0; i < 8; ++i) CK_CHECK(choice8[i] >= -1 && choice8[i] <= 5, CKKS_EINVAL, "variant must be -1..5");
        for (int i = 0; i < 8; ++i) ctx->ntt_choice[i] = choice8[i];
    });
}

// ---------------------------------------------------------------- keys ------
int ckks_keygen(ckks_ctx* ctx, const int32_t* steps, int n, int want_conj, ckks_keys** out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(out);
        CK_CHECK(n == 0 || steps, CKKS_EINVAL, "rot_steps is NULL");
        *out = ops::keygen(ctx, steps, n, want_conj);
    });
}

int ckks_keys_add_rotations(ckks_ctx* ctx, ckks_keys* keys, const int32_t* steps, int n) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(keys);
        for (int i = 0; i < n; ++i) ops::add_galois_key(ctx, *keys, ops::galois_of_step(ctx, steps[i]));
    });
}

int ckks_keys_destroy(ckks_keys* keys) {
    delete keys;
    return CKKS_OK;
}

int ckks_keys_export_secret(ckks_ctx* ctx, const ckks_keys* keys, int64_t* s) {
    return guard(ctx, [&] {
        REQ(keys);
        REQ(s);
        std::copy(keys->s.begin(), keys->s.end(), s);
    });
}

// -------------------------------------------------------------- handles -----
int ckks_ct_create(ckks_ctx* ctx, ckks_ct** out) {
    if (!ctx || !out) return CKKS_EINVAL;
    *out = new ckks_ct();
    (*out)->ctx = ctx;
    return CKKS_OK;
}
int ckks_ct_destroy(ckks_ct* ct) {
    delete ct;
    return CKKS_OK;
}
int ckks_ct_info(const ckks_ct* ct, int* level, double* scale) {
    if (!ct) return CKKS_EINVAL;
    if (level) *level = ct->level;
    if (scale) *scale = ct->scale;
    return CKKS_OK;
}
int ckks_ct_set_scale(ckks_ct* ct, double scale) {
    if (!ct) return CKKS_EINVAL;
    ct->scale = scale;
    return CKKS_OK;
}

int ckks_ct_import_rns(ckks_ctx* ctx, const uint64_t* host, int level, double scale, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(host);
        REQ(out);
        CK_CHECK(level >= 0 && level <= ctx->L, CKKS_EINVAL, "level out of range");
        ckks_ct o = ops::new_ct(ctx, level, scale);
        const size_t words = 2 * (size_t)(level + 1) * ctx->n;
        CUDA_CHECK(cudaMemcpyAsync(o.buf.ptr, host, words * 8, cudaMemcpyHostToDevice, ctx->stream));
        kern::ntt_forward(ctx, o.buf.ptr, 2 * (level + 1), ctx->d_iota, level + 1);
        assign(out, std::move(o));
    });
}

int ckks_ct_copy_into(ckks_ctx* ctx, const ckks_ct* src, ckks_ct* dst) {
    return guard(ctx, [&] {
        CT_OK(src);
        CT_OK(dst);
        CK_CHECK(src->level == dst->level, CKKS_EINVAL, "copy_into needs equal levels");
        if (src == dst) return;
        CUDA_CHECK(cudaMemcpyAsync(dst->buf.ptr, src->buf.ptr, 2 * (size_t)(src->level + 1) * ctx->n * 8,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
        dst->scale = src->scale;
    });
}

int ckks_ct_export_rns(ckks_ctx* ctx, const ckks_ct* ct, uint64_t* host) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(ct);
        REQ(host);
        CK_CHECK(ct->level >= 0, CKKS_EINVAL, "empty ciphertext");
        const int nl = ct->level + 1;
        const size_t words = 2 * (size_t)nl * ctx->n;
        DevBuf t(words, ctx->stream);
        kern::ntt_inverse_from(ctx, ct->buf.ptr, (size_t)nl * ctx->n, t.ptr, 2 * nl, ctx->d_iota, nl, 0, nullptr);
        CUDA_CHECK(cudaMemcpyAsync(host, t.ptr, words * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    });
}

int ckks_pt_create(ckks_ctx* ctx, ckks_pt** out) {
    if (!ctx || !out) return CKKS_EINVAL;
    *out = new ckks_pt();
    (*out)->ctx = ctx;
    return CKKS_OK;
}
int ckks_pt_destroy(ckks_pt* pt) {
    delete pt;
    return CKKS_OK;
}
int ckks_pt_info(const ckks_pt* pt, int* level, double* scale) {
    if (!pt) return CKKS_EINVAL;
    if (level) *level = pt->level;
    if (scale) *scale = pt->scale;
    return CKKS_OK;
}

int ckks_pt_import_rns(ckks_ctx* ctx, const uint64_t* host, int level, double scale, ckks_pt* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(host);
        REQ(out);
        CK_CHECK(level >= 0 && level <= ctx->L, CKKS_EINVAL, "level out of range");
        const size_t words = (size_t)(level + 1) * ctx->n;
        DevBuf b(words, ctx->stream);
        CUDA_CHECK(cudaMemcpyAsync(b.ptr, host, words * 8, cudaMemcpyHostToDevice, ctx->stream));
        kern::ntt_forward(ctx, b.ptr, level + 1, ctx->d_iota, level + 1);
        out->ctx = ctx;
        out->buf = std::move(b);
        out->level = level;
        out->scale = scale;
    });
}

int ckks_pt_export_rns(ckks_ctx* ctx, const ckks_pt* pt, uint64_t* host) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(pt);
        REQ(host);
        const size_t words = (size_t)(pt->level + 1) * ctx->n;
        DevBuf t(words, ctx->stream);
        CUDA_CHECK(cudaMemcpyAsync(t.ptr, pt->buf.ptr, words * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        kern::ntt_inverse(ctx, t.ptr, pt->level + 1, ctx->d_iota, pt->level + 1);
        CUDA_CHECK(cudaMemcpyAsync(host, t.ptr, words * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    });
}

// ------------------------------------------------------------- encoding -----
int ckks_encode(ckks_ctx* ctx, const double* re, const double* im, int n, int level, double scale, int kind,
                int slice_len, ckks_pt* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(re);
        REQ(out);
        const int N = ctx->n;
        if (kind == CKKS_SLOT) {
            CK_CHECK(n >= 0 && n <= N / 2, CKKS_EINVAL, "too many slots");
            std::vector<cplx> z(N / 2, cplx(0, 0));
            for (int j = 0; j < n; ++j) z[j] = cplx(re[j], im ? im[j] : 0.0);
            encode_complex(ctx, z, level, scale, out);
        } else if (kind == CKKS_COEFF) {
            CK_CHECK(n >= 0 && n <= N, CKKS_EINVAL, "too many coefficients");
            std::vector<double> f(N, 0.0);
            for (int j = 0; j < n; ++j) f[j] = re[j];
            CK_CHECK(level >= 0 && level <= ctx->L, CKKS_EINVAL, "level out of range");
            upload_coeffs(ctx, round_coeffs(f, scale), level, scale, out);
        } else if (kind == CKKS_CINS_REAL) {
            CK_CHECK(slice_len >= 2 && (slice_len & (slice_len - 1)) == 0 && slice_len <= N, CKKS_EINVAL,
                     "slice_len must be a power of two in [2, N]");
            const int C = N / slice_len;
            CK_CHECK(n >= 0 && n <= N, CKKS_EINVAL, "too many values");
            std::vector<double> m(N, 0.0);
            for (int j = 0; j < n; ++j) m[j] = re[j];
            encode_complex(ctx, fp64::real_cins_slots(m.data(), C, slice_len), level, scale, out);
        } else {
            CK_THROW(CKKS_EINVAL, "unknown encoding kind");
        }
    });
}

int ckks_decode(ckks_ctx* ctx, const ckks_pt* pt, int kind, int slice_len, double* re, double* im, int n) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(pt);
        REQ(re);
        const int N = ctx->n;
        const int nl = pt->level + 1;
        DevBuf t((size_t)nl * N, ctx->stream);
        CUDA_CHECK(cudaMemcpyAsync(t.ptr, pt->buf.ptr, (size_t)nl * N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        kern::ntt_inverse(ctx, t.ptr, nl, ctx->d_iota, nl);
        std::vector<u64> h = download(ctx, t.ptr, (size_t)nl * N);
        std::vector<double> f = crt_centred(ctx, h, nl);
        for (double& x : f) x /= pt->scale;
        if (kind == CKKS_COEFF) {
            CK_CHECK(n <= N, CKKS_EINVAL, "n above N");
            for (int j = 0; j < n; ++j) re[j] = f[j];
        } else if (kind == CKKS_SLOT) {
            CK_CHECK(n <= N / 2, CKKS_EINVAL, "n above N/2");
            std::vector<cplx> z = fp64::decode_slots(f, N);
            for (int j = 0; j < n; ++j) {
                re[j] = z[j].real();
                if (im) im[j] = z[j].imag();
            }
        } else if (kind == CKKS_CINS_REAL) {
            CK_CHECK(slice_len >= 2 && (slice_len & (slice_len - 1)) == 0 && slice_len <= N, CKKS_EINVAL,
                     "bad slice_len");
            std::vector<double> m = fp64::cins_to_reals(fp64::decode_slots(f, N), N / slice_len, slice_len);
            for (int j = 0; j < n && j < N; ++j) re[j] = m[j];
        } else {
            CK_THROW(CKKS_EINVAL, "unknown encoding kind");
        }
    });
}

int ckks_encode_image(ckks_ctx* ctx, const double* img, int c, int w0, int w, int level, double scale,
                      ckks_pt* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(img);
        REQ(out);
        const int N = ctx->n;
        CK_CHECK(w >= 2 && (w & (w - 1)) == 0 && w * w <= N && w0 >= 1 && w0 <= w, CKKS_EINVAL, "bad w / w0");
        const int two_l = w * w, C = N / two_l;
        CK_CHECK(c >= 1 && c <= C, CKKS_EINVAL, "channels do not fit in one ciphertext");
        std::vector<double> m(N, 0.0);
        for (int i = 0; i < c; ++i)
            for (int r = 0; r < w0; ++r)
                for (int col = 0; col < w0; ++col)
                    m[(size_t)i * two_l + r * w + col] = img[((size_t)i * w0 + r) * w0 + col];
        encode_complex(ctx, fp64::real_cins_slots(m.data(), C, two_l), level, scale, out);
    });
}

int ckks_decode_image(ckks_ctx* ctx, const ckks_pt* pt, int from_coeff, int c, int w0, int w, double* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(pt);
        REQ(out);
        const int N = ctx->n;
        CK_CHECK(w >= 2 && (w & (w - 1)) == 0 && w * w <= N && w0 >= 1 && w0 <= w, CKKS_EINVAL, "bad w / w0");
        const int two_l = w * w, C = N / two_l;
        CK_CHECK(c >= 1 && c <= C, CKKS_EINVAL, "channels do not fit in one ciphertext");
        const int nl = pt->level + 1;
        DevBuf t((size_t)nl * N, ctx->stream);
        CUDA_CHECK(cudaMemcpyAsync(t.ptr, pt->buf.ptr, (size_t)nl * N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        kern::ntt_inverse(ctx, t.ptr, nl, ctx->d_iota, nl);
        std::vector<double> f = crt_centred(ctx, download(ctx, t.ptr, (size_t)nl * N), nl);
        for (double& x : f) x /= pt->scale;
        int cbits = 0;
        while ((1 << cbits) < C) ++cbits;
        std::vector<double> m;
        if (!from_coeff) m = fp64::cins_to_reals(fp64::decode_slots(f, N), C, two_l);
        for (int i = 0; i < c; ++i) {
            unsigned rv = 0, x = (unsigned)i;
            for (int b = 0; b < cbits; ++b) {
                rv = (rv << 1) | (x & 1);
                x >>= 1;
            }
            for (int r = 0; r < w0; ++r)
                for (int col = 0; col < w0; ++col) {
                    const int k = r * w + col;
                    out[((size_t)i * w0 + r) * w0 + col] =
                        from_coeff ? f[(size_t)k * C + rv] : m[(size_t)i * two_l + k];
                }
        }
    });
}

// ----------------------------------------------------------- encryption -----
int ckks_encrypt(ckks_ctx* ctx, const ckks_keys* keys, const ckks_pt* pt, uint64_t nonce, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        REQ(pt);
        REQ(out);
        CK_CHECK(pt->level >= 0, CKKS_EINVAL, "empty plaintext");
        assign(out, ops::encrypt(*keys, *pt, nonce));
    });
}
int ckks_encrypt_sk(ckks_ctx* ctx, const ckks_keys* keys, const ckks_pt* pt, uint64_t nonce, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        REQ(pt);
        REQ(out);
        CK_CHECK(pt->level >= 0, CKKS_EINVAL, "empty plaintext");
        assign(out, ops::encrypt_sk(*keys, *pt, nonce));
    });
}
int ckks_decrypt(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* ct, ckks_pt* out) {
    return guard(ctx, [&] {
        REQ(keys);
        REQ(ct);
        REQ(out);
        ops::decrypt(*keys, *ct, *out);
    });
}

// -------------------------------------------------------------- HE ops ------

int ckks_add(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(a);
        CT_OK(b);
        REQ(out);
        assign(out, ops::add(*a, *b));
    });
}
int ckks_sub(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(a);
        CT_OK(b);
        REQ(out);
        assign(out, ops::sub(*a, *b));
    });
}
int ckks_mul_plain(ckks_ctx* ctx, const ckks_ct* ct, const ckks_pt* pt, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(ct);
        REQ(pt);
        REQ(out);
        assign(out, ops::mul_plain(*ct, *pt));
    });
}
int ckks_mul_relin(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* a, const ckks_ct* b, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        CT_OK(a);
        CT_OK(b);
        REQ(out);
        assign(out, ops::mul_relin(*keys, *a, *b));
    });
}
int ckks_mul_int(ckks_ctx* ctx, const ckks_ct* ct, int64_t c, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(ct);
        REQ(out);
        assign(out, ops::mul_int(*ct, c));
    });
}
int ckks_add_const(ckks_ctx* ctx, const ckks_ct* ct, double c, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(ct);
        REQ(out);
        assign(out, ops::add_const(*ct, c));
    });
}
int ckks_imult(ckks_ctx* ctx, const ckks_ct* ct, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(ct);
        REQ(out);
        assign(out, ops::imult(*ct));
    });
}
int ckks_rescale(ckks_ctx* ctx, const ckks_ct* ct, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(ct);
        REQ(out);
        assign(out, ops::rescale(*ct));
    });
}
int ckks_mod_drop(ckks_ctx* ctx, const ckks_ct* ct, int level, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(ct);
        REQ(out);
        assign(out, ops::mod_drop(*ct, level));
    });
}
int ckks_level_down(ckks_ctx* ctx, const ckks_ct* ct, int level, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(ct);
        REQ(out);
        assign(out, ops::level_down(*ct, level));
    });
}
int ckks_mod_raise(ckks_ctx* ctx, const ckks_ct* ct, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(ct);
        REQ(out);
        assign(out, ops::mod_raise(*ct));
    });
}
int ckks_rotate_hoisted(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const int32_t* steps, int n,
                        ckks_ct* const* outs) {
    return guard(ctx, [&] {
        REQ(keys);
        CT_OK(in);
        CK_CHECK(n >= 0 && (n == 0 || (steps && outs)), CKKS_EINVAL, "bad steps/outs");
        for (int i = 0; i < n; ++i) CK_CHECK(outs[i] && outs[i] != in, CKKS_EINVAL, "outs must not alias the input");
        std::vector<long long> st(steps, steps + n);
        std::vector<ckks_ct> r = ops::rotate_hoisted(*keys, *in, st);
        for (int i = 0; i < n; ++i) assign(outs[i], std::move(r[i]));
    });
}
int ckks_conjugate(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* ct, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        CT_OK(ct);
        REQ(out);
        assign(out, ops::conjugate(*keys, *ct));
    });
}

// ----------------------------------------------------------------- BSGS -----
int ckks_ptset_create(ckks_ctx* ctx, int a0, int step, int count, int B, int level, double scale, ckks_ptset** out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(out);
        CK_CHECK(step >= 1 && count >= 1 && level >= 0 && level <= ctx->L, CKKS_EINVAL, "bad plan parameters");
        const int m = ctx->n / 2;
        ckks_ptset* ps = new ckks_ptset();
        ps->ctx = ctx;
        ps->a0 = ((a0 % m) + m) % m;
        ps->step = step;
        ps->count = count;
        ps->B = B > 0 ? B : fp64::default_bsgs_B(count);
        ps->level = level;
        ps->scale = scale;
        *out = ps;
    });
}
int ckks_ptset_destroy(ckks_ptset* ps) {
    delete ps;
    return CKKS_OK;
}
int ckks_ptset_set_rns(ckks_ctx* ctx, ckks_ptset* ps, int g, int b, const uint64_t* host) {
    return guard(ctx, [&] {
        REQ(ps);
        REQ(host);
        CK_CHECK(g >= 0 && g < ps->G() && b >= 0 && b < ps->B && g * ps->B + b < ps->count, CKKS_EINVAL,
                 "(g, b) outside the plan");
        // limbs over Q_level u P, coefficient domain
        const int rows = ps->level + 1 + ctx->np;
        auto pt = std::make_unique<ckks_pt>();
        DevBuf buf((size_t)rows * ctx->n, ctx->stream);
        CUDA_CHECK(cudaMemcpyAsync(buf.ptr, host, (size_t)rows * ctx->n * 8, cudaMemcpyHostToDevice, ctx->stream));
        kern::ntt_forward(ctx, buf.ptr, rows, ctx->d_ext_ids[ps->level], rows);
        pt->ctx = ctx;
        pt->buf = std::move(buf);
        pt->level = ps->level;
        pt->scale = ps->scale;
        pt->ext = true;
        ps->pts[std::make_pair(g, b)] = std::move(pt);
    });
}
int ckks_ptset_info(const ckks_ptset* ps, int* a0, int* step, int* count, int* B, int* level, double* scale,
                    int* n_pts) {
    if (!ps) return CKKS_EINVAL;
    if (a0) *a0 = ps->a0;
    if (step) *step = ps->step;
    if (count) *count = ps->count;
    if (B) *B = ps->B;
    if (level) *level = ps->level;
    if (scale) *scale = ps->scale;
    if (n_pts) *n_pts = (int)ps->pts.size();
    return CKKS_OK;
}

static void plan_rotations(const ckks_ptset& ps, std::set<int>& out) {
    const long long m = ps.ctx->n / 2;
    for (const auto& kv : ps.pts) {
        long long b = (long long)ps.step * kv.first.second % m;
        if (b) out.insert((int)b);
        long long R = ((long long)ps.a0 + (long long)ps.step * kv.first.first * ps.B) % m;
        if (R) out.insert((int)R);
    }
}

int ckks_ptset_rotations(const ckks_ptset* ps, int32_t* steps, int cap, int* n_out) {
    if (!ps || !n_out) return CKKS_EINVAL;
    std::set<int> s;
    plan_rotations(*ps, s);
    int i = 0;
    for (int r : s) {
        if (steps && i < cap) steps[i] = r;
        ++i;
    }
    *n_out = i;
    return CKKS_OK;
}

int ckks_bsgs(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* ct, const ckks_ptset* ps, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        CT_OK(ct);
        REQ(ps);
        REQ(out);
        assign(out, ops::bsgs(*keys, *ct, *ps));
    });
}

int ckks_ptset_conv_fused(ckks_ctx* ctx, const double* W, int cin, int cout, int f, int w, int level,
                          double pt_scale, int B, ckks_ptset** out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(W);
        REQ(out);
        CK_CHECK(w >= 2 && (w & (w - 1)) == 0 && w * w <= ctx->n, CKKS_EINVAL, "w must be a power of two, w^2 <= N");
        CK_CHECK(f >= 1 && f % 2 == 1 && f <= w, CKKS_EINVAL, "kernel size must be odd and <= w");
        CK_CHECK(level >= 1 && level <= ctx->L, CKKS_EINVAL, "the fused conv needs level >= 1");
        const int two_l = w * w, ell = two_l / 2, C = ctx->n / two_l, m = ctx->n / 2;
        std::vector<std::vector<cplx>> diags = fp64::fused_conv_diagonals(W, cin, cout, f, w, ctx->n);
        fp64::Diag D;
        for (int d = 0; d < C; ++d) {
            double mx = 0;
            for (const cplx& v : diags[d]) mx = std::max(mx, std::abs(v));
            if (mx > 0) D[(int)(((long long)d * ell) % m)] = diags[d];
        }
        *out = make_plan(ctx, D, 0, ell, C, level, pt_scale, B);
    });
}

int ckks_ptset_conv_fused_s2(ckks_ctx* ctx, const double* W, int cin, int cout, int f, int w_in, int t, int level,
                             double pt_scale, int B, ckks_ptset** out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(W);
        REQ(out);
        CK_CHECK(w_in >= 4 && (w_in & (w_in - 1)) == 0 && w_in * w_in <= ctx->n, CKKS_EINVAL,
                 "w_in must be a power of two, 4 <= w_in, w_in^2 <= N");
        CK_CHECK(f >= 1 && f % 2 == 1, CKKS_EINVAL, "kernel size must be odd");
        const int C = ctx->n / (w_in * w_in), w = w_in / 2;
        CK_CHECK(t >= 0 && t * C < cin, CKKS_EINVAL, "input ciphertext index out of range");
        CK_CHECK(cout >= 1 && cout <= 4 * C, CKKS_EINVAL, "more output channels than slices");
        CK_CHECK(level >= 1 && level <= ctx->L, CKKS_EINVAL, "the fused conv needs level >= 1");
        int fo = 0;
        std::vector<double> Wd = fp64::decompose_kernels(W, cout, cin, f, C, t, &fo);
        CK_CHECK(fo <= w, CKKS_EINVAL, "decomposed kernel wider than the output image");
        const int two_l = w * w, ell = two_l / 2, Cn = ctx->n / two_l, m = ctx->n / 2;
        std::vector<std::vector<cplx>> diags = fp64::fused_conv_diagonals(Wd.data(), 4 * C, cout, fo, w, ctx->n);
        fp64::Diag D;
        for (int d = 0; d < Cn; ++d) {
            double mx = 0;
            for (const cplx& v : diags[d]) mx = std::max(mx, std::abs(v));
            if (mx > 0) D[(int)(((long long)d * ell) % m)] = diags[d];
        }
        *out = make_plan(ctx, D, 0, ell, Cn, level, pt_scale, B);
    });
}

// Downsampling depthwise conv (Sec. 3.3.4): output channel o reads input channel o only, so
// the kernels form a diagonal W[o][o] = K[o] of the stride-2 conv above.
int ckks_ptset_dwconv_fused_s2(ckks_ctx* ctx, const double* K, int c, int f, int w_in, int t, int level,
                               double pt_scale, int B, ckks_ptset** out) {
    std::vector<double> W;
    const int st = guard(ctx, [&] {
        REQ(ctx);
        REQ(K);
        CK_CHECK(c >= 1 && f >= 1 && (long long)c * c * f * f <= (1LL << 28), CKKS_EINVAL,
                 "channel count or kernel size out of range");
        W.assign((size_t)c * c * f * f, 0.0);
        for (int o = 0; o < c; ++o)
            std::copy(K + (size_t)o * f * f, K + (size_t)(o + 1) * f * f, W.begin() + ((size_t)o * c + o) * f * f);
    });
    if (st != CKKS_OK) return st;
    return ckks_ptset_conv_fused_s2(ctx, W.data(), c, c, f, w_in, t, level, pt_scale, B, out);
}

int ckks_ptset_fc_stoc(ckks_ctx* ctx, const double* M, int n_out, int n_in, int level, double pt_scale, int B,
                       ckks_ptset** out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(M);
        REQ(out);
        const int m = ctx->n / 2;
        CK_CHECK(n_in >= 1 && n_in <= m && (n_in & (n_in - 1)) == 0, CKKS_EINVAL, "n_in must be a power of two <= N/2");
        CK_CHECK(n_out >= 1 && n_out <= m, CKKS_EINVAL, "n_out must be in [1, N/2]");
        CK_CHECK(level >= 1 && level <= ctx->L, CKKS_EINVAL, "the fused FC needs level >= 1");
        *out = make_plan(ctx, fp64::fc_stoc_diagonals(M, n_out, n_in, ctx->n), 0, 1, n_in, level, pt_scale, B);
    });
}

int ckks_fc_stoc(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const ckks_ptset* fc, int n_in, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        CT_OK(in);
        REQ(fc);
        REQ(out);
        const int m = ctx->n / 2;
        CK_CHECK(n_in >= 1 && n_in <= m && (n_in & (n_in - 1)) == 0 && fc->count == n_in, CKKS_EINVAL,
                 "n_in must be the plaintext set's diagonal count, a power of two");
        ckks_ct x = ops::copy_ct(*in);
        for (int s = n_in; s < m; s *= 2) x = ops::add(x, ops::rotate(*keys, x, -s));
        assign(out, ops::bsgs(*keys, x, *fc, true));
    });
}

int ckks_ptset_decompose(ckks_ctx* ctx, int w, int level, double scale, int B, ckks_ptset** out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(out);
        CK_CHECK(w >= 4 && (w & (w - 1)) == 0 && w * w <= ctx->n, CKKS_EINVAL, "w must be a power of two, 4 <= w");
        CK_CHECK(level >= 1 && level <= ctx->L, CKKS_EINVAL, "bad level");
        *out = make_plan(ctx, fp64::decompose_diag(w, ctx->n / 2), (1 - w) * (w / 4), w / 4, 2 * w - 1, level, scale,
                         B);
    });
}

int ckks_encode_dwconv_kernel(ckks_ctx* ctx, const double* K, int c, int f, int w, int level, double scale,
                              ckks_pt* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(K);
        REQ(out);
        CK_CHECK(w >= 2 && (w & (w - 1)) == 0 && w * w <= ctx->n, CKKS_EINVAL, "w must be a power of two, w^2 <= N");
        CK_CHECK(f >= 1 && f % 2 == 1 && f <= w, CKKS_EINVAL, "kernel size must be odd and <= w");
        encode_complex(ctx, fp64::dwconv_kernel_slots(K, c, f, w, ctx->n), level, scale, out);
    });
}

int ckks_dwconv_cins(ckks_ctx* ctx, const ckks_ct* in, const ckks_pt* kernel, ckks_ct* out) {
    return guard(ctx, [&] {
        CT_OK(in);
        REQ(kernel);
        REQ(out);
        assign(out, ops::rescale(ops::mul_plain(*in, *kernel)));
    });
}

int ckks_conv2d_cins(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const ckks_ptset* conv, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        CT_OK(in);
        REQ(conv);
        REQ(out);
        assign(out, ops::bsgs(*keys, *in, *conv, true));
    });
}

// -------------------------------------------------------- bootstrapping -----
// diagonals of one BSGS level of a bootstrapping configuration
static fp64::Diag boot_level_diag(const ckks_boot& bt, const ckks_boot::Level& lv, int m) {
    if (lv.kind == 1) return fp64::decompose_diag(bt.bp.w, m);
    std::vector<int> rev(lv.strides.rbegin(), lv.strides.rend());
    fp64::Diag D = fp64::s_product(rev, m, lv.kind == 0);
    if (lv.half)
        for (auto& kv : D)
            for (cplx& v : kv.second) v *= 0.5;
    return D;
}

static std::unique_ptr<ckks_ptset>& boot_level_slot(ckks_boot& bt, const ckks_boot::Level& lv) {
    if (lv.kind == 0) return bt.ctos[lv.index];
    if (lv.kind == 1) return bt.decomp;
    return bt.stoc[lv.index];
}

static std::unique_ptr<ckks_ptset> boot_level_plan(ckks_ctx* ctx, const ckks_boot& bt, const ckks_boot::Level& lv,
                                                   int B) {
    return std::unique_ptr<ckks_ptset>(make_plan(ctx, boot_level_diag(bt, lv, ctx->n / 2), lv.a0, lv.step, lv.count,
                                                 lv.level, lv.scale, B));
}

int ckks_boot_create(ckks_ctx* ctx, const ckks_boot_params* bp, ckks_boot** out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(bp);
        REQ(out);
        CK_CHECK(bp->w >= 2 && (bp->w & (bp->w - 1)) == 0 && bp->w * bp->w <= ctx->n, CKKS_EINVAL, "bad w");
        CK_CHECK(bp->K >= 1 && bp->r >= 0 && bp->deg >= 2 && bp->ctos_levels >= 1 && bp->stoc_levels >= 1,
                 CKKS_EINVAL, "bad bootstrapping parameters");
        std::unique_ptr<ckks_boot> bt(new ckks_boot());
        bt->ctx = ctx;
        bt->bp = *bp;
        const int n = ctx->n, m = n / 2, L = ctx->L;
        bt->two_l = bp->w * bp->w;
        bt->ell = bt->two_l / 2;
        bt->C = n / bt->two_l;
        const double q0 = (double)ctx->q[0];
        const int ld = L - bp->ctos_levels;
        CK_CHECK(ld >= 2, CKKS_ELEVEL, "not enough levels for CtoS");
        bt->l_drop = ld;
        bt->c_drop = llround_away((ctx->delta[ld - 1] * (double)ctx->q[ld]) / (q0 * (double)bp->K));
        CK_CHECK(bt->c_drop >= 1, CKKS_EINVAL, "scale-drop constant below 1");
        bt->K_eff = (ctx->delta[ld - 1] * (double)ctx->q[ld]) / (q0 * (double)bt->c_drop);
        bt->s_raise = q0 * bt->K_eff;
        // CtoS = T^{-1}: stages N/4 ... 1, largest stride first
        std::vector<int> stages;
        for (int k = m / 2; k >= 1; k /= 2) stages.push_back(k);
        std::vector<std::vector<int>> groups = fp64::split_groups(stages, bp->ctos_levels);
        bt->ctos.resize(groups.size());
        for (size_t i = 0; i < groups.size(); ++i) {
            ckks_boot::Level lv;
            lv.kind = 0;
            lv.index = (int)i;
            lv.strides = groups[i];
            lv.half = i + 1 == groups.size();
            fp64::ap_of_group(groups[i], m, &lv.a0, &lv.step, &lv.count);
            lv.level = L - (int)i;
            lv.scale = (double)ctx->q[lv.level];
            bt->ctos[i] = boot_level_plan(ctx, *bt, lv, fp64::boot_bsgs_B(lv.count));
            bt->levels.push_back(lv);
        }
        bt->coeffs = fp64::cheb_interp_cos(bt->K_eff, bp->r, bp->deg);
        int depth = 0;
        while ((1 << depth) < bp->deg) ++depth;
        bt->l_em = (ld - 1) - (depth + 1) - bp->r;
        CK_CHECK(bt->l_em - 1 - bp->stoc_levels >= 0, CKKS_ELEVEL, "not enough levels for the block");
        const int le = bt->l_em;
        bt->s_em = (ctx->delta[le + 1] * ctx->delta[le + 1]) / (double)ctx->q[le + 1];
        bt->s_mask = (ctx->delta[le - 1] * (double)ctx->q[le]) / bt->s_em;
        // padding masks times q0 / (2 pi delta0): slot i l + u carries pixel rev_l(u) (Re) or rev_l(u) + l (Im)
        const double val = q0 / (2.0 * 3.14159265358979323846 * bp->delta0);
        std::vector<cplx> mre(m, cplx(0, 0)), mim(m, cplx(0, 0));
        int lbits = 0;
        while ((1 << lbits) < bt->ell) ++lbits;
        for (int i = 0; i < bp->cout && i < bt->C; ++i)
            for (int u = 0; u < bt->ell; ++u) {
                unsigned k = 0, x = u;
                for (int b = 0; b < lbits; ++b) {
                    k = (k << 1) | (x & 1);
                    x >>= 1;
                }
                int p1 = (int)k, p2 = (int)k + bt->ell;
                if (p1 / bp->w < bp->w0 && p1 % bp->w < bp->w0) mre[(size_t)i * bt->ell + u] = val;
                if (p2 / bp->w < bp->w0 && p2 % bp->w < bp->w0) mim[(size_t)i * bt->ell + u] = val;
            }
        bt->mask_im_zero = std::all_of(mim.begin(), mim.end(), [](const cplx& v) { return v == cplx(0, 0); });
        bt->mask_re = std::make_unique<ckks_pt>();
        bt->mask_im = std::make_unique<ckks_pt>();
        encode_complex(ctx, mre, le, bt->s_mask, bt->mask_re.get());
        encode_complex(ctx, mim, le, bt->s_mask, bt->mask_im.get());
        // stride 2 (Alg. 2): the decomposition at canonical scale, then StoC1 over slices of l/4
        CK_CHECK(bp->stride == 0 || bp->stride == 1 || bp->stride == 2, CKKS_EINVAL, "stride must be 1 or 2");
        int top = le - 1, ell_out = bt->ell;
        if (bp->stride == 2) {
            CK_CHECK(bp->w >= 4 && bp->w0 % 2 == 0, CKKS_EINVAL, "stride 2 needs w >= 4 and an even image width");
            ckks_boot::Level lv;
            lv.kind = 1;
            lv.a0 = (1 - bp->w) * (bp->w / 4);
            lv.step = bp->w / 4;
            lv.count = 2 * bp->w - 1;
            lv.level = top;
            lv.scale = ctx->delta[top];
            bt->decomp = boot_level_plan(ctx, *bt, lv, fp64::boot_bsgs_B(lv.count));
            bt->levels.push_back(lv);
            --top;
            ell_out /= 4;
        }
        // StoC1 = S_{l' <- 1}: stages 1, 2, ..., l'/2, smallest stride first
        std::vector<int> st;
        for (int k = 1; k < ell_out; k *= 2) st.push_back(k);
        std::vector<std::vector<int>> sg = fp64::split_groups(st, bp->stoc_levels);
        bt->stoc.resize(sg.size());
        for (size_t i = 0; i < sg.size(); ++i) {
            ckks_boot::Level lv;
            lv.kind = 2;
            lv.index = (int)i;
            lv.strides = sg[i];
            fp64::ap_of_group(sg[i], m, &lv.a0, &lv.step, &lv.count);
            lv.level = top - (int)i;
            lv.scale = ctx->delta[lv.level];
            bt->stoc[i] = boot_level_plan(ctx, *bt, lv, fp64::boot_bsgs_B(lv.count));
            bt->levels.push_back(lv);
        }
        bt->l_out = top - (int)bt->stoc.size();
        CK_CHECK(bt->l_out >= 1, CKKS_ELEVEL, "not enough levels for the block");
        *out = bt.release();
    });
}

int ckks_boot_destroy(ckks_boot* bt) {
    delete bt;
    return CKKS_OK;
}

int ckks_boot_info(const ckks_boot* bt, double* info) {
    if (!bt || !info) return CKKS_EINVAL;
    info[0] = bt->K_eff;
    info[1] = bt->s_raise;
    info[2] = (double)bt->c_drop;
    info[3] = bt->l_drop;
    info[4] = bt->l_em;
    info[5] = bt->l_out;
    info[6] = bt->s_em;
    info[7] = bt->s_mask;
    return CKKS_OK;
}

int ckks_boot_rotations(const ckks_boot* bt, int32_t* steps, int cap, int* n_out) {
    if (!bt || !n_out) return CKKS_EINVAL;
    std::set<int> s;
    for (const auto& p : bt->ctos) plan_rotations(*p, s);
    for (const auto& p : bt->stoc) plan_rotations(*p, s);
    if (bt->decomp) plan_rotations(*bt->decomp, s);
    int i = 0;
    for (int r : s) {
        if (steps && i < cap) steps[i] = r;
        ++i;
    }
    *n_out = i;
    return CKKS_OK;
}

int ckks_boot_bsgs_splits(const ckks_boot* bt, int32_t* B, int cap, int* n_out) {
    if (!bt || !n_out) return CKKS_EINVAL;
    int i = 0;
    for (const auto& lv : bt->levels) {
        const ckks_ptset* p = lv.kind == 0 ? bt->ctos[lv.index].get()
                              : lv.kind == 1 ? bt->decomp.get() : bt->stoc[lv.index].get();
        if (B && i < cap) B[i] = p ? p->B : 0;
        ++i;
    }
    *n_out = i;
    return CKKS_OK;
}

int ckks_boot_set_bsgs_splits(ckks_ctx* ctx, ckks_boot* bt, const int32_t* B, int n) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(bt);
        CK_CHECK(n == (int)bt->levels.size() && (n == 0 || B), CKKS_EINVAL, "one baby-step count per BSGS level");
        for (int i = 0; i < n; ++i)
            CK_CHECK(B[i] >= 1 && B[i] <= kern::BsgsGiants::MAXB, CKKS_EINVAL, "baby-step count out of range");
        for (int i = 0; i < n; ++i) boot_level_slot(*bt, bt->levels[i]) = boot_level_plan(ctx, *bt, bt->levels[i], B[i]);
    });
}

// For every BSGS level: candidate baby-step counts (powers of two up to 32 and the cost-model
// choice), each timed as one HMatmul with rescale on a fresh encryption at the level's input
// level, with switching keys generated for the candidates' rotations only while the level is
// tuned; the fastest plan is kept.  Op and launch counters are left as they were.
int ckks_boot_tune_bsgs(ckks_ctx* ctx, ckks_boot* bt, int reps, int32_t* B_out, int cap, int* n_out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(bt);
        CK_CHECK(reps >= 1, CKKS_EINVAL, "reps must be >= 1");
        const auto ops_saved = ctx->ops;
        const long long launches_saved = ctx->launches;
        cudaEvent_t e0, e1;
        CUDA_CHECK(cudaEventCreate(&e0));
        CUDA_CHECK(cudaEventCreate(&e1));
        std::vector<int> chosen;
        for (const auto& lv : bt->levels) {
            std::vector<int> cand;
            for (int b = 2; b <= std::min(lv.count, kern::BsgsGiants::MAXB); b *= 2) cand.push_back(b);
            const int def = fp64::boot_bsgs_B(lv.count);
            if (std::find(cand.begin(), cand.end(), def) == cand.end()) cand.push_back(def);
            if (cand.size() < 2) {
                chosen.push_back(boot_level_slot(*bt, lv)->B);
                continue;
            }
            std::vector<std::unique_ptr<ckks_ptset>> plans;
            std::set<int> rots;
            for (int b : cand) {
                plans.push_back(boot_level_plan(ctx, *bt, lv, b));
                plan_rotations(*plans.back(), rots);
            }
            std::vector<int32_t> steps(rots.begin(), rots.end());
            std::unique_ptr<ckks_keys> keys(ops::keygen(ctx, steps.data(), (int)steps.size(), 0));
            ckks_pt pt;
            encode_complex(ctx, std::vector<cplx>(ctx->n / 2, cplx(0, 0)), lv.level, ctx->delta[lv.level], &pt);
            const ckks_ct x = ops::encrypt(*keys, pt, 1);
            int best = -1;
            float best_ms = 0;
            for (size_t k = 0; k < plans.size(); ++k) {
                ops::bsgs(*keys, x, *plans[k], true);      // warm-up
                CUDA_CHECK(cudaEventRecord(e0, ctx->stream));
                for (int r = 0; r < reps; ++r) ops::bsgs(*keys, x, *plans[k], true);
                CUDA_CHECK(cudaEventRecord(e1, ctx->stream));
                CUDA_CHECK(cudaEventSynchronize(e1));
                float ms = 0;
                CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
                if (best < 0 || ms < best_ms) {
                    best = (int)k;
                    best_ms = ms;
                }
            }
            chosen.push_back(plans[best]->B);
            boot_level_slot(*bt, lv) = std::move(plans[best]);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ctx->ops = ops_saved;
        ctx->launches = launches_saved;
        for (size_t i = 0; i < chosen.size(); ++i)
            if (B_out && (int)i < cap) B_out[i] = chosen[i];
        if (n_out) *n_out = (int)chosen.size();
    });
}

static std::unique_ptr<ckks_ptset> clone_ptset(ckks_ctx* ctx, const ckks_ptset& ps) {
    auto o = std::make_unique<ckks_ptset>();
    o->ctx = ctx;
    o->a0 = ps.a0;
    o->step = ps.step;
    o->count = ps.count;
    o->B = ps.B;
    o->level = ps.level;
    o->scale = ps.scale;
    for (const auto& kv : ps.pts) {
        auto pt = std::make_unique<ckks_pt>();
        const size_t words = (size_t)(kv.second->level + 1 + (kv.second->ext ? ctx->np : 0)) * ctx->n;
        pt->ctx = ctx;
        pt->buf = DevBuf(words, ctx->stream);
        pt->level = kv.second->level;
        pt->scale = kv.second->scale;
        pt->ext = kv.second->ext;
        CUDA_CHECK(cudaMemcpyAsync(pt->buf.ptr, kv.second->buf.ptr, words * 8, cudaMemcpyDeviceToDevice,
                                   ctx->stream));
        o->pts[kv.first] = std::move(pt);
    }
    return o;
}

int ckks_boot_set_ctos(ckks_ctx* ctx, ckks_boot* bt, int i, const ckks_ptset* ps) {
    return guard(ctx, [&] {
        REQ(bt);
        REQ(ps);
        CK_CHECK(i >= 0 && i < (int)bt->ctos.size() && ps->level == bt->ctos[i]->level, CKKS_EINVAL,
                 "bad CtoS index or level");
        bt->ctos[i] = clone_ptset(ctx, *ps);
    });
}
int ckks_boot_set_stoc(ckks_ctx* ctx, ckks_boot* bt, int i, const ckks_ptset* ps) {
    return guard(ctx, [&] {
        REQ(bt);
        REQ(ps);
        CK_CHECK(i >= 0 && i < (int)bt->stoc.size() && ps->level == bt->stoc[i]->level, CKKS_EINVAL,
                 "bad StoC index or level");
        bt->stoc[i] = clone_ptset(ctx, *ps);
    });
}
int ckks_boot_set_decomp(ckks_ctx* ctx, ckks_boot* bt, const ckks_ptset* ps) {
    return guard(ctx, [&] {
        REQ(bt);
        REQ(ps);
        CK_CHECK(bt->decomp && ps->level == bt->decomp->level, CKKS_EINVAL, "no decomposition at that level");
        bt->decomp = clone_ptset(ctx, *ps);
    });
}
int ckks_boot_set_coeffs(ckks_ctx* ctx, ckks_boot* bt, const double* c, int deg) {
    return guard(ctx, [&] {
        REQ(bt);
        REQ(c);
        CK_CHECK(deg == bt->bp.deg, CKKS_EINVAL, "degree differs from the configuration");
        bt->coeffs.assign(c, c + deg + 1);
    });
}
int ckks_boot_set_masks(ckks_ctx* ctx, ckks_boot* bt, const ckks_pt* re, const ckks_pt* im) {
    return guard(ctx, [&] {
        REQ(bt);
        REQ(re);
        REQ(im);
        CK_CHECK(re->level == bt->l_em && im->level == bt->l_em, CKKS_EINVAL, "masks must sit at l_em");
        for (int k = 0; k < 2; ++k) {
            const ckks_pt* src = k ? im : re;
            auto pt = std::make_unique<ckks_pt>();
            const size_t words = (size_t)(src->level + 1) * ctx->n;
            pt->ctx = ctx;
            pt->buf = DevBuf(words, ctx->stream);
            pt->level = src->level;
            pt->scale = src->scale;
            CUDA_CHECK(cudaMemcpyAsync(pt->buf.ptr, src->buf.ptr, words * 8, cudaMemcpyDeviceToDevice, ctx->stream));
            (k ? bt->mask_im : bt->mask_re) = std::move(pt);
        }
        std::vector<u64> h = download(ctx, bt->mask_im->buf.ptr, (size_t)(bt->mask_im->level + 1) * ctx->n);
        bt->mask_im_zero = std::all_of(h.begin(), h.end(), [](u64 v) { return v == 0; });
    });
}

int ckks_bootstrap(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* bt, const ckks_ct* ct0, ckks_ct* out_re,
                   ckks_ct* out_im) {
    return guard(ctx, [&] {
        REQ(keys);
        REQ(bt);
        CT_OK(ct0);
        REQ(out_re);
        REQ(out_im);
        ckks_ct re, im;
        ops::bootstrap(*keys, *bt, *ct0, re, im);
        assign(out_re, std::move(re));
        assign(out_im, std::move(im));
    });
}

int ckks_stoc1(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* re, const ckks_ct* im, const ckks_boot* bt,
               ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        CT_OK(re);
        CT_OK(im);
        REQ(bt);
        REQ(out);
        assign(out, ops::stoc1(*keys, *bt, *re, *im));
    });
}

int ckks_block(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const ckks_ptset* conv, const ckks_boot* bt,
               ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        CT_OK(in);
        REQ(conv);
        REQ(bt);
        REQ(out);
        assign(out, ops::block(*keys, *bt, *conv, *in));
    });
}

int ckks_block_multi(ckks_ctx* ctx, const ckks_keys* keys, int n_in, const ckks_ct* const* in,
                     const ckks_ptset* const* conv, const ckks_boot* bt, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        REQ(in);
        REQ(conv);
        REQ(bt);
        REQ(out);
        CK_CHECK(n_in >= 1 && n_in <= 64, CKKS_EINVAL, "n_in must be in [1, 64]");
        std::vector<const ckks_ct*> ins;
        std::vector<const ckks_ptset*> convs;
        for (int t = 0; t < n_in; ++t) {
            CT_OK(in[t]);
            REQ(conv[t]);
            CK_CHECK(in[t]->level == in[0]->level && in[t]->scale == in[0]->scale, CKKS_EINVAL,
                     "input ciphertexts differ in level or scale");
            CK_CHECK(conv[t]->level == conv[0]->level && conv[t]->scale == conv[0]->scale, CKKS_EINVAL,
                     "conv plaintext sets differ in level or scale");
            ins.push_back(in[t]);
            convs.push_back(conv[t]);
        }
        assign(out, ops::block_multi(*keys, *bt, convs, ins));
    });
}

}  // extern "C"

struct ckks_graph {
    ckks_ctx* ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    ~ckks_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

// Runs `run` once eagerly (sizing `out`, building lazily created tables), then records a
// second run on the context's stream and a copy of its result into out's buffer.  The
// temporaries of the recorded run are allocated and freed inside the graph.
template <class F>
static void capture_graph(ckks_ctx* ctx, ckks_ct* out, ckks_graph** g, F run) {
    CK_CHECK(ctx->stream != nullptr, CKKS_EINVAL, "graphs need a context created on a non-default stream");
    assign(out, run());
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    std::unique_ptr<ckks_graph> gr(new ckks_graph());
    gr->ctx = ctx;
    const long long l0 = ctx->launches;
    CUDA_CHECK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    try {
        ckks_ct r = run();
        CK_CHECK(r.level == out->level, CKKS_EINVAL, "captured run changed level");
        CUDA_CHECK(cudaMemcpyAsync(out->buf.ptr, r.buf.ptr, 2 * (size_t)(r.level + 1) * ctx->n * 8,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
    } catch (...) {
        cudaGraph_t tmp = nullptr;
        cudaStreamEndCapture(ctx->stream, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
        throw;
    }
    CUDA_CHECK(cudaStreamEndCapture(ctx->stream, &gr->graph));
    CUDA_CHECK(cudaGraphInstantiate(&gr->exec, gr->graph, 0));
    gr->launches = ctx->launches - l0;
    *g = gr.release();
}

// checks of the downsampling layer's arguments; fills the pointer lists
static void ds_args(int n_in, const ckks_ct* const* re, const ckks_ct* const* im, const ckks_ptset* const* conv,
                    const ckks_boot* bt_in, const ckks_boot* bt_out, std::vector<const ckks_ct*>& vre,
                    std::vector<const ckks_ct*>& vim, std::vector<const ckks_ptset*>& vconv) {
    REQ(re);
    REQ(im);
    REQ(conv);
    REQ(bt_in);
    REQ(bt_out);
    CK_CHECK(n_in >= 1 && n_in <= 64, CKKS_EINVAL, "n_in must be in [1, 64]");
    CK_CHECK(bt_in->bp.stride == 2, CKKS_EINVAL, "bt_in must be a stride-2 configuration");
    for (int t = 0; t < n_in; ++t) {
        CT_OK(re[t]);
        CT_OK(im[t]);
        REQ(conv[t]);
        CK_CHECK(conv[t]->level == conv[0]->level && conv[t]->scale == conv[0]->scale, CKKS_EINVAL,
                 "conv plaintext sets differ in level or scale");
        vre.push_back(re[t]);
        vim.push_back(im[t]);
        vconv.push_back(conv[t]);
    }
}

extern "C" {

int ckks_block_graph_create(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const ckks_ptset* conv,
                            const ckks_boot* bt, ckks_ct* out, ckks_graph** g) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(keys);
        CT_OK(in);
        REQ(conv);
        REQ(bt);
        REQ(out);
        REQ(g);
        CK_CHECK(out != in, CKKS_EINVAL, "out must not alias in");
        capture_graph(ctx, out, g, [&] { return ops::block(*keys, *bt, *conv, *in); });
    });
}

int ckks_downsample_layer(ckks_ctx* ctx, const ckks_keys* keys, int n_in, const ckks_ct* const* re,
                          const ckks_ct* const* im, const ckks_boot* bt_in, const ckks_ptset* const* conv,
                          const ckks_boot* bt_out, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        REQ(out);
        std::vector<const ckks_ct*> vre, vim;
        std::vector<const ckks_ptset*> vconv;
        ds_args(n_in, re, im, conv, bt_in, bt_out, vre, vim, vconv);
        assign(out, ops::downsample_layer(*keys, *bt_in, *bt_out, vre, vim, vconv));
    });
}

int ckks_downsample_layer_graph_create(ckks_ctx* ctx, const ckks_keys* keys, int n_in, const ckks_ct* const* re,
                                       const ckks_ct* const* im, const ckks_boot* bt_in,
                                       const ckks_ptset* const* conv, const ckks_boot* bt_out, ckks_ct* out,
                                       ckks_graph** g) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(keys);
        REQ(out);
        REQ(g);
        std::vector<const ckks_ct*> vre, vim;
        std::vector<const ckks_ptset*> vconv;
        ds_args(n_in, re, im, conv, bt_in, bt_out, vre, vim, vconv);
        for (int t = 0; t < n_in; ++t) CK_CHECK(out != re[t] && out != im[t], CKKS_EINVAL, "out must not alias an input");
        capture_graph(ctx, out, g, [&] { return ops::downsample_layer(*keys, *bt_in, *bt_out, vre, vim, vconv); });
    });
}

// ---- lockstep batches: B ciphertexts of one shape through one block, every kernel launched once
// for all of them (keys and plaintext diagonals read once per launch) ----
namespace {
// the inputs gathered into one batched ciphertext [B][2][l+1][N]
ckks_ct gather_batch(ckks_ctx* ctx, int B, const ckks_ct* const* in) {
    CK_CHECK(B >= 1 && B <= 1024, CKKS_EINVAL, "B must be in [1, 1024]");
    REQ(in);
    for (int t = 0; t < B; ++t) {
        CT_OK(in[t]);
        CK_CHECK(in[t]->nb == 1 && in[t]->level == in[0]->level, CKKS_EINVAL, "batch inputs differ in level");
        CK_CHECK(fabs(in[t]->scale - in[0]->scale) <= ldexp(1.0, -30) * fabs(in[0]->scale), CKKS_EINVAL,
                 "batch inputs differ in scale");
    }
    ckks_ct x = ops::new_ct(ctx, in[0]->level, in[0]->scale, B);
    for (int t = 0; t < B; ++t)
        CUDA_CHECK(cudaMemcpyAsync(x.c0(t), in[t]->buf.ptr, x.cstride() * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    return x;
}
// each ciphertext of a batch into its own handle (sized before, when `sized`)
void scatter_batch(ckks_ctx* ctx, const ckks_ct& y, ckks_ct* const* out, bool sized) {
    for (int t = 0; t < y.nb; ++t) {
        if (!sized) ops::ensure_ct(*out[t], ctx, y.level);
        CK_CHECK(out[t]->level == y.level && out[t]->nb == 1, CKKS_EINVAL, "output handle changed shape");
        out[t]->scale = y.scale;
        CUDA_CHECK(cudaMemcpyAsync(out[t]->buf.ptr, y.c0(t), y.cstride() * 8, cudaMemcpyDeviceToDevice,
                                   ctx->stream));
    }
}
void batch_args(int B, const ckks_ct* const* in, ckks_ct* const* out) {
    REQ(in);
    REQ(out);
    for (int t = 0; t < B; ++t) {
        REQ(out[t]);
        for (int u = 0; u < B; ++u) CK_CHECK(out[t] != in[u], CKKS_EINVAL, "outputs must not alias inputs");
        for (int u = 0; u < t; ++u) CK_CHECK(out[t] != out[u], CKKS_EINVAL, "outputs must be distinct");
    }
}
}  // namespace

int ckks_block_batched(ckks_ctx* ctx, const ckks_keys* keys, int B, const ckks_ct* const* in,
                       const ckks_ptset* conv, const ckks_boot* bt, ckks_ct* const* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(keys);
        REQ(conv);
        REQ(bt);
        batch_args(B, in, out);
        ckks_ct x = gather_batch(ctx, B, in);
        ckks_ct y = ops::block(*keys, *bt, *conv, x);
        scatter_batch(ctx, y, out, false);
    });
}

int ckks_block_batched_graph_create(ckks_ctx* ctx, const ckks_keys* keys, int B, const ckks_ct* const* in,
                                    const ckks_ptset* conv, const ckks_boot* bt, ckks_ct* const* out,
                                    ckks_graph** g) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(keys);
        REQ(conv);
        REQ(bt);
        REQ(g);
        batch_args(B, in, out);
        CK_CHECK(ctx->stream != nullptr, CKKS_EINVAL, "graphs need a context created on a non-default stream");
        {   // one eager run: sizes the outputs and builds any lazily created table
            ckks_ct x = gather_batch(ctx, B, in);
            scatter_batch(ctx, ops::block(*keys, *bt, *conv, x), out, false);
        }
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        std::unique_ptr<ckks_graph> gr(new ckks_graph());
        gr->ctx = ctx;
        const long long l0 = ctx->launches;
        CUDA_CHECK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        try {
            ckks_ct x = gather_batch(ctx, B, in);
            scatter_batch(ctx, ops::block(*keys, *bt, *conv, x), out, true);
        } catch (...) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(ctx->stream, &tmp);
            if (tmp) cudaGraphDestroy(tmp);
            throw;
        }
        CUDA_CHECK(cudaStreamEndCapture(ctx->stream, &gr->graph));
        CUDA_CHECK(cudaGraphInstantiate(&gr->exec, gr->graph, 0));
        gr->launches = ctx->launches - l0;
        *g = gr.release();
    });
}

int ckks_downsample_layer_batched(ckks_ctx* ctx, const ckks_keys* keys, int B, int n_in, const ckks_ct* const* re,
                                  const ckks_ct* const* im, const ckks_boot* bt_in, const ckks_ptset* const* conv,
                                  const ckks_boot* bt_out, ckks_ct* const* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(keys);
        REQ(re);
        REQ(im);
        REQ(out);
        CK_CHECK(B >= 1 && B <= 1024, CKKS_EINVAL, "B must be in [1, 1024]");
        std::vector<const ckks_ct*> vre, vim;
        std::vector<const ckks_ptset*> vconv;
        ds_args(n_in, re, im, conv, bt_in, bt_out, vre, vim, vconv);     // checks input 0's n_in pairs
        std::vector<ckks_ct> R, I;
        std::vector<const ckks_ct*> col(B);
        for (int t = 0; t < n_in; ++t) {
            for (int b = 0; b < B; ++b) col[b] = re[(size_t)b * n_in + t];
            R.push_back(gather_batch(ctx, B, col.data()));
            for (int b = 0; b < B; ++b) col[b] = im[(size_t)b * n_in + t];
            I.push_back(gather_batch(ctx, B, col.data()));
        }
        for (int b = 0; b < B; ++b) {
            REQ(out[b]);
            for (int u = 0; u < B * n_in; ++u)
                CK_CHECK(out[b] != re[u] && out[b] != im[u], CKKS_EINVAL, "outputs must not alias inputs");
        }
        std::vector<const ckks_ct*> pr, pi;
        for (int t = 0; t < n_in; ++t) {
            pr.push_back(&R[t]);
            pi.push_back(&I[t]);
        }
        scatter_batch(ctx, ops::downsample_layer(*keys, *bt_in, *bt_out, pr, pi, vconv), out, false);
    });
}

int ckks_bootstrap_batched(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* bt, int B, const ckks_ct* const* in,
                           ckks_ct* const* out_re, ckks_ct* const* out_im) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(keys);
        REQ(bt);
        batch_args(B, in, out_re);
        batch_args(B, in, out_im);
        for (int b = 0; b < B; ++b)
            for (int u = 0; u < B; ++u) CK_CHECK(out_re[b] != out_im[u], CKKS_EINVAL, "outputs must be distinct");
        ckks_ct x = gather_batch(ctx, B, in);
        ckks_ct re, im;
        ops::bootstrap(*keys, *bt, x, re, im);
        scatter_batch(ctx, re, out_re, false);
        scatter_batch(ctx, im, out_im, false);
    });
}

int ckks_eval_poly_batched(ckks_ctx* ctx, const ckks_keys* keys, int B, const ckks_ct* const* in,
                           const double* coeffs, int deg, int basis, double a, double b, ckks_ct* const* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(keys);
        REQ(coeffs);
        batch_args(B, in, out);
        CK_CHECK(basis == CKKS_BASIS_CHEB || basis == CKKS_BASIS_POWER, CKKS_EINVAL, "unknown basis");
        CK_CHECK(deg >= 1, CKKS_EINVAL, "polynomial degree must be >= 1");
        CK_CHECK(std::isfinite(a) && std::isfinite(b) && b > a, CKKS_EINVAL, "the interval needs a < b");
        ckks_ct x = gather_batch(ctx, B, in);
        std::vector<double> c(coeffs, coeffs + deg + 1);
        scatter_batch(ctx, ops::eval_poly(*keys, x, c, basis == CKKS_BASIS_POWER, a, b), out, false);
    });
}

int ckks_eval_relu_batched(ckks_ctx* ctx, const ckks_keys* keys, int B, const ckks_ct* const* in,
                           const double* coeffs, const int* degs, int n_stages, ckks_ct* const* out) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(keys);
        REQ(coeffs);
        REQ(degs);
        batch_args(B, in, out);
        CK_CHECK(n_stages >= 1, CKKS_EINVAL, "n_stages must be >= 1");
        std::vector<std::vector<double>> st;
        size_t off = 0;
        for (int i = 0; i < n_stages; ++i) {
            CK_CHECK(degs[i] >= 1, CKKS_EINVAL, "stage degree must be >= 1");
            st.emplace_back(coeffs + off, coeffs + off + degs[i] + 1);
            off += degs[i] + 1;
        }
        ckks_ct x = gather_batch(ctx, B, in);
        scatter_batch(ctx, ops::eval_relu(*keys, x, st), out, false);
    });
}

int ckks_graph_launch(ckks_graph* g, void* stream) {
    if (!g) return CKKS_EINVAL;
    return guard(g->ctx, [&] {
        CUDA_CHECK(cudaGraphLaunch(g->exec, stream ? (cudaStream_t)stream : g->ctx->stream));
        g->ctx->launches += g->launches;
    });
}

int ckks_graph_info(const ckks_graph* g, int64_t* kernel_launches) {
    if (!g) return CKKS_EINVAL;
    if (kernel_launches) *kernel_launches = g->launches;
    return CKKS_OK;
}

int ckks_graph_destroy(ckks_graph* g) {
    delete g;
    return CKKS_OK;
}

// Batched blocks: one recorded block per input, the graphs spread over streams of their own
// so that independent ciphertexts overlap on the device; fork and join through events on
// the context's stream.
struct ckks_batch {
    ckks_ctx* ctx = nullptr;
    std::vector<ckks_graph*> graphs;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;      // one per stream
    cudaEvent_t fork = nullptr;
    ~ckks_batch() {
        for (ckks_graph* g : graphs) delete g;
        for (cudaEvent_t e : done) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        for (cudaStream_t s : streams) cudaStreamDestroy(s);
    }
};

int ckks_block_batch_create(ckks_ctx* ctx, const ckks_keys* keys, int B, const ckks_ct* const* in,
                            const ckks_ptset* conv, const ckks_boot* bt, ckks_ct* const* out, int n_streams,
                            ckks_batch** batch) {
    return guard(ctx, [&] {
        REQ(ctx);
        REQ(in);
        REQ(out);
        REQ(batch);
        CK_CHECK(B >= 1 && B <= 1024, CKKS_EINVAL, "batch size must be 1..1024");
        CK_CHECK(n_streams >= 1 && n_streams <= 32, CKKS_EINVAL, "stream count must be 1..32");
        for (int i = 0; i < B; ++i) {
            CT_OK(in[i]);
            REQ(out[i]);
            for (int j = 0; j < B; ++j) {
                CK_CHECK(out[i] != in[j], CKKS_EINVAL, "an output aliases an input of the batch");
                CK_CHECK(j == i || out[i] != out[j], CKKS_EINVAL, "outputs of the batch must be distinct");
            }
        }
        std::unique_ptr<ckks_batch> b(new ckks_batch);
        b->ctx = ctx;
        for (int i = 0; i < B; ++i) {
            ckks_graph* g = nullptr;
            const int st = ckks_block_graph_create(ctx, keys, in[i], conv, bt, out[i], &g);
            if (st != CKKS_OK) CK_THROW(st, ctx->err);
            b->graphs.push_back(g);
        }
        const int S = std::min(n_streams, B);
        for (int k = 0; k < S; ++k) {
            cudaStream_t s = nullptr;
            CUDA_CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            b->streams.push_back(s);
            cudaEvent_t e = nullptr;
            CUDA_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            b->done.push_back(e);
        }
        CUDA_CHECK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        *batch = b.release();
    });
}

int ckks_batch_launch(ckks_batch* b) {
    if (!b) return CKKS_EINVAL;
    return guard(b->ctx, [&] {
        ckks_ctx* c = b->ctx;
        const size_t S = b->streams.size();
        CUDA_CHECK(cudaEventRecord(b->fork, c->stream));
        for (cudaStream_t s : b->streams) CUDA_CHECK(cudaStreamWaitEvent(s, b->fork, 0));
        for (size_t i = 0; i < b->graphs.size(); ++i) {
            CUDA_CHECK(cudaGraphLaunch(b->graphs[i]->exec, b->streams[i % S]));
            c->launches += b->graphs[i]->launches;
        }
        for (size_t k = 0; k < S; ++k) {
            CUDA_CHECK(cudaEventRecord(b->done[k], b->streams[k]));
            CUDA_CHECK(cudaStreamWaitEvent(c->stream, b->done[k], 0));
        }
    });
}

int ckks_batch_destroy(ckks_batch* b) {
    if (b) {
        cudaStreamSynchronize(b->ctx->stream);     // the graphs may still run
        delete b;
    }
    return CKKS_OK;
}

int ckks_eval_poly(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const double* coeffs, int deg, int basis,
                   double a, double b, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        CT_OK(in);
        REQ(coeffs);
        REQ(out);
        CK_CHECK(basis == CKKS_BASIS_CHEB || basis == CKKS_BASIS_POWER, CKKS_EINVAL, "unknown basis");
        CK_CHECK(deg >= 1, CKKS_EINVAL, "polynomial degree must be >= 1");
        CK_CHECK(std::isfinite(a) && std::isfinite(b) && b > a, CKKS_EINVAL, "the interval needs a < b");
        std::vector<double> c(coeffs, coeffs + deg + 1);
        assign(out, ops::eval_poly(*keys, *in, c, basis == CKKS_BASIS_POWER, a, b));
    });
}

int ckks_eval_relu(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, const double* coeffs, const int* degs,
                   int n_stages, ckks_ct* out) {
    return guard(ctx, [&] {
        REQ(keys);
        CT_OK(in);
        REQ(coeffs);
        REQ(degs);
        REQ(out);
        CK_CHECK(n_stages >= 1, CKKS_EINVAL, "n_stages must be >= 1");
        std::vector<std::vector<double>> st;
        size_t off = 0;
        for (int i = 0; i < n_stages; ++i) {
            CK_CHECK(degs[i] >= 1, CKKS_EINVAL, "stage degree must be >= 1");
            st.emplace_back(coeffs + off, coeffs + off + degs[i] + 1);
            off += degs[i] + 1;
        }
        assign(out, ops::eval_relu(*keys, *in, st));
    });
}

// ------------------------------------------------------------ raw NTT -------
static int raw_ntt(ckks_ctx* ctx, uint64_t* dev, int n_limbs, const int32_t* ids, bool inv) {
    return guard(ctx, [&] {
        REQ(ctx);
        CK_CHECK(n_limbs >= 0, CKKS_EINVAL, "negative limb count");
        if (n_limbs == 0) return;      // nothing to transform (dev and ids may be NULL)
        REQ(dev);
        REQ(ids);
        for (int i = 0; i < n_limbs; ++i)
            CK_CHECK(ids[i] >= 0 && ids[i] < ctx->nall, CKKS_EINVAL, "prime id out of range");
        std::vector<u64> tmp(n_limbs);
        DevBuf d((n_limbs + 1) / 2, ctx->stream);
        std::vector<int> v(ids, ids + n_limbs);
        CUDA_CHECK(cudaMemcpyAsync(d.ptr, v.data(), n_limbs * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        if (inv)
            kern::ntt_inverse(ctx, (u64*)dev, n_limbs, (const int*)d.ptr, n_limbs);
        else
            kern::ntt_forward(ctx, (u64*)dev, n_limbs, (const int*)d.ptr, n_limbs);
    });
}
int ckks_ntt_forward(ckks_ctx* ctx, uint64_t* dev, int n_limbs, const int32_t* ids) {
    return raw_ntt(ctx, dev, n_limbs, ids, false);
}
int ckks_ntt_inverse(ckks_ctx* ctx, uint64_t* dev, int n_limbs, const int32_t* ids) {
    return raw_ntt(ctx, dev, n_limbs, ids, true);
}

}  // extern "C"
