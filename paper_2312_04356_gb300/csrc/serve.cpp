// Serving loop: continuous batching of inference requests over a fixed set of slots.
//
// A model is a chain of Alg. 1 blocks.  For every (slot, model) pair the whole request --
// import of the client's coefficient-domain limbs (NTT), the blocks (with a level drop to the
// next conv's level between them), export (iNTT) -- is recorded once as a CUDA graph that
// reads the slot's device input buffer and writes its device output buffer; the temporaries
// are allocated and freed inside the graph.  A worker thread admits queued requests, in
// submission order, into free slots while the bytes of temporaries held by the requests in
// flight stay within the HBM budget, and retires them as their slot's stream completes, so
// requests join and leave the running set one at a time (no batch barrier).  Keys, plaintext
// sets and bootstrapping tables stay resident and are shared by every slot.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>

#include "ckks.h"
#include "internal.h"
#include "scheme_ops.h"

#define REQ(p) CK_CHECK((p) != nullptr, CKKS_EINVAL, #p " is NULL")

namespace {

using Clock = std::chrono::steady_clock;

// One layer of a model: n_out output ciphertexts from n_in inputs, output j from k of them
// (in_index).  A block layer computes each output as an Alg. 1 block over its inputs (ckks_block, or the Sec. 3.3.3 block matrix-vector
// product when n_in > 1); a downsampling layer (Alg. 2) computes each output from the EvalMod
// outputs of the layer before it, which then stops after its bootstrap (no StoC1).
struct Layer {
    int kind = CKKS_LAYER_BLOCK;
    int n_in = 1, n_out = 1, k = 1;
    std::vector<int> in_index;              // [n_out][k] (every output reads inputs 0..n_in-1 if empty)
    std::vector<const ckks_ptset*> convs;   // [n_out][k]
    const ckks_boot* boot = nullptr;        // block: its configuration; downsampling: bt_out
    const ckks_boot* boot_in = nullptr;     // downsampling: bt_in (stride-2 tail of the inputs)
};

struct Model {
    std::vector<Layer> layers;
    int in_level = 0, out_level = 0;
    double in_scale = 0, out_scale = 0;
    int n_in = 1, n_out = 1;      // ciphertexts into and out of a request
    long long footprint = 0;      // peak bytes of temporaries of one request
    long long kernels = 0;        // kernel launches of one request's graph
    size_t in_words(size_t n) const { return (size_t)n_in * 2 * (size_t)(in_level + 1) * n; }
    size_t out_words(size_t n) const { return (size_t)n_out * 2 * (size_t)(out_level + 1) * n; }
};

struct Request {
    uint64_t id = 0;
    int model = 0;
    int state = CKKS_REQ_QUEUED;
    bool cancel = false;
    std::vector<u64> in, out;
    Clock::time_point t_submit, t_done;
    std::string err;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    // by model: coefficient-domain input and output limbs and their pinned staging; each model's
    // recorded graphs read and write its own buffers, which live as long as the server
    std::vector<u64*> d_in, d_out, h_in, h_out;
    std::vector<cudaGraphExec_t> exec;   // by model
    std::vector<cudaGraph_t> graph;
    uint64_t req = 0;             // 0: free
};

}  // namespace

struct ckks_server {
    ckks_ctx* ctx = nullptr;
    const ckks_keys* keys = nullptr;
    ckks_server_params sp{};
    int device = 0;
    std::vector<Model> models;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    long long in_use = 0;         // footprint of the requests in flight
    int in_flight = 0, max_in_flight = 0;
    long long completed = 0, failed = 0, cancelled = 0, kernels = 0;
    std::vector<double> lat_ms;
    std::thread worker;
    bool started = false, stop = false;
    std::string err;
    ~ckks_server();
};

namespace {

template <class F>
int sguard(ckks_server* s, F&& f) {
    try {
        f();
        return CKKS_OK;
    } catch (const CkksError& e) {
        if (s) s->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (s) s->err = "host allocation failed";
        return CKKS_ENOMEM;
    } catch (const std::exception& e) {
        if (s) s->err = e.what();
        return CKKS_EINVAL;
    }
}

// One request of model m, reading d_in and writing d_out (both coefficient domain,
// [ciphertexts][2][level + 1][N]).
void run_model(ckks_server* s, const Model& m, const u64* d_in, u64* d_out) {
    ckks_ctx* c = s->ctx;
    const ckks_keys& keys = *s->keys;
    const size_t per_in = 2 * (size_t)(m.in_level + 1) * c->n;
    std::vector<ckks_ct> xs;
    for (int i = 0; i < m.n_in; ++i) {
        ckks_ct x = ops::new_ct(c, m.in_level, m.in_scale);
        CUDA_CHECK(cudaMemcpyAsync(x.buf.ptr, d_in + i * per_in, per_in * 8, cudaMemcpyDeviceToDevice, c->stream));
        kern::ntt_forward(c, x.buf.ptr, 2 * (m.in_level + 1), c->d_iota, m.in_level + 1);
        xs.push_back(std::move(x));
    }
    std::vector<ckks_ct> res, ims;    // EvalMod outputs handed to a downsampling layer
    for (size_t k = 0; k < m.layers.size(); ++k) {
        const Layer& L = m.layers[k];
        const bool to_ds = k + 1 < m.layers.size() && m.layers[k + 1].kind == CKKS_LAYER_DOWNSAMPLE;
        std::vector<ckks_ct> ys, nre, nim;
        if (L.kind == CKKS_LAYER_BLOCK) {
            const int lev = L.convs[0]->level;
            for (ckks_ct& x : xs)
                if (x.level != lev) x = ops::level_down(x, lev);
            for (int j = 0; j < L.n_out; ++j) {
                const std::vector<const ckks_ptset*> cs(L.convs.begin() + (size_t)j * L.k,
                                                        L.convs.begin() + (size_t)(j + 1) * L.k);
                std::vector<const ckks_ct*> ins;
                for (int t = 0; t < L.k; ++t) ins.push_back(&xs[L.in_index.empty() ? t : L.in_index[j * L.k + t]]);
                if (!to_ds) {
                    ys.push_back(L.n_in == 1 ? ops::block(keys, *L.boot, *cs[0], *ins[0])
                                             : ops::block_multi(keys, *L.boot, cs, ins));
                } else {
                    const ckks_ct x0 = L.n_in == 1 ? ops::bsgs(keys, *ins[0], *cs[0], true)
                                                   : ops::bsgs_multi(keys, ins, cs, true);
                    ckks_ct re, im;
                    ops::bootstrap(keys, *L.boot, x0, re, im);
                    nre.push_back(std::move(re));
                    nim.push_back(std::move(im));
                }
            }
        } else {
            for (int j = 0; j < L.n_out; ++j) {
                const std::vector<const ckks_ptset*> cs(L.convs.begin() + (size_t)j * L.k,
                                                        L.convs.begin() + (size_t)(j + 1) * L.k);
                std::vector<const ckks_ct*> rp, ip;
                for (int t = 0; t < L.k; ++t) {
                    const int i = L.in_index.empty() ? t : L.in_index[j * L.k + t];
                    rp.push_back(&res[i]);
                    ip.push_back(&ims[i]);
                }
                ys.push_back(ops::downsample_layer(keys, *L.boot_in, *L.boot, rp, ip, cs));
            }
        }
        xs = std::move(ys);
        res = std::move(nre);
        ims = std::move(nim);
    }
    const size_t per_out = 2 * (size_t)(m.out_level + 1) * c->n;
    for (int j = 0; j < m.n_out; ++j) {
        CK_CHECK(xs[j].level == m.out_level, CKKS_EINVAL, "model output level changed");
        const int nl = m.out_level + 1;
        kern::ntt_inverse_from(c, xs[j].buf.ptr, (size_t)nl * c->n, d_out + j * per_out, 2 * nl, c->d_iota, nl, 0,
                               nullptr);
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double r = p * (double)(v.size() - 1);
    const size_t i = (size_t)r;
    const double f = r - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

// Retire finished slots, then (unless stopping) admit queued requests.  Called with
// s->mu held.  Returns whether requests are in flight.
bool step(ckks_server* s) {
    bool busy = false;
    for (Slot& sl : s->slots) {
        if (!sl.req) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) {
            busy = true;
            continue;
        }
        Request& r = s->reqs[sl.req];
        r.t_done = Clock::now();
        if (q != cudaSuccess) {
            r.state = CKKS_REQ_FAILED;
            r.err = cudaGetErrorString(q);
            ++s->failed;
        } else if (r.cancel) {
            r.state = CKKS_REQ_CANCELLED;
            ++s->cancelled;
        } else {
            r.out.assign(sl.h_out[r.model], sl.h_out[r.model] + s->models[r.model].out_words(s->ctx->n));
            r.state = CKKS_REQ_DONE;
            ++s->completed;
            s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
        }
        r.in.clear();
        r.in.shrink_to_fit();
        s->in_use -= s->models[r.model].footprint;
        --s->in_flight;
        sl.req = 0;
        s->cv_done.notify_all();
    }
    while (!s->stop && !s->queue.empty()) {
        const uint64_t id = s->queue.front();
        Request& r = s->reqs[id];
        if (r.cancel) {
            r.state = CKKS_REQ_CANCELLED;
            ++s->cancelled;
            s->queue.pop_front();
            s->cv_done.notify_all();
            continue;
        }
        const Model& m = s->models[r.model];
        if (s->sp.hbm_budget > 0 && s->in_use + m.footprint > s->sp.hbm_budget) break;
        Slot* free_slot = nullptr;
        for (Slot& sl : s->slots)
            if (!sl.req) {
                free_slot = &sl;
                break;
            }
        if (!free_slot) break;
        s->queue.pop_front();
        Slot& sl = *free_slot;
        std::copy(r.in.begin(), r.in.end(), sl.h_in[r.model]);
        cudaError_t e = cudaMemcpyAsync(sl.d_in[r.model], sl.h_in[r.model], r.in.size() * 8, cudaMemcpyHostToDevice,
                                        sl.stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec[r.model], sl.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.h_out[r.model], sl.d_out[r.model], m.out_words(s->ctx->n) * 8,
                                cudaMemcpyDeviceToHost, sl.stream);
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
        if (e != cudaSuccess) {
            r.state = CKKS_REQ_FAILED;
            r.err = cudaGetErrorString(e);
            r.t_done = Clock::now();
            ++s->failed;
            s->cv_done.notify_all();
            continue;
        }
        r.state = CKKS_REQ_RUNNING;
        sl.req = id;
        s->in_use += m.footprint;
        s->kernels += m.kernels;
        s->max_in_flight = std::max(s->max_in_flight, ++s->in_flight);
        busy = true;
    }
    return busy;
}

void worker_main(ckks_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        const bool busy = step(s);
        if (s->stop && s->in_flight == 0) break;     // queued requests are abandoned
        if (busy)
            s->cv.wait_for(lk, std::chrono::microseconds(50));   // poll the slots' events
        else
            s->cv.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    }
}

}  // namespace

ckks_server::~ckks_server() {
    {
        std::lock_guard<std::mutex> lk(mu);
        stop = true;
    }
    cv.notify_all();
    if (worker.joinable()) worker.join();
    for (Slot& sl : slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        for (cudaGraphExec_t e : sl.exec)
            if (e) cudaGraphExecDestroy(e);
        for (cudaGraph_t g : sl.graph)
            if (g) cudaGraphDestroy(g);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        for (u64* p : sl.d_in) cudaFree(p);
        for (u64* p : sl.d_out) cudaFree(p);
        for (u64* p : sl.h_in) cudaFreeHost(p);
        for (u64* p : sl.h_out) cudaFreeHost(p);
    }
}

extern "C" {

int ckks_server_create(ckks_ctx* ctx, const ckks_keys* keys, const ckks_server_params* sp, ckks_server** out) {
    if (!ctx || !keys || !sp || !out) return CKKS_EINVAL;
    if (sp->slots < 1 || sp->slots > 64 || sp->hbm_budget < 0) return CKKS_EINVAL;
    std::unique_ptr<ckks_server> s(new ckks_server());
    return sguard(s.get(), [&] {
        CK_CHECK(ctx->stream != nullptr, CKKS_EINVAL, "the server records graphs: the context needs a non-default stream");
        s->ctx = ctx;
        s->keys = keys;
        s->sp = *sp;
        CUDA_CHECK(cudaGetDevice(&s->device));
        s->slots.resize(sp->slots);
        for (Slot& sl : s->slots) {
            CUDA_CHECK(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
            CUDA_CHECK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
        }
        *out = s.release();
    });
}

}  // extern "C"

namespace {

// checks a model's layers, sizes the slots' buffers, runs one request eagerly (checking keys and
// levels, measuring the footprint) and records the request's graph for every slot
void add_model_impl(ckks_server* s, Model m, int* model_id) {
    CK_CHECK(!s->started, CKKS_EINVAL, "models are added before ckks_server_start");
    CK_CHECK(!s->ctx->timing, CKKS_EINVAL, "switch kernel timing off before recording graphs");
    ckks_ctx* c = s->ctx;
    const int nl = (int)m.layers.size();
    CK_CHECK(nl >= 1 && nl <= 64, CKKS_EINVAL, "a model has 1 to 64 layers");
    for (int k = 0; k < nl; ++k) {
        const Layer& L = m.layers[k];
        CK_CHECK(L.kind == CKKS_LAYER_BLOCK || L.kind == CKKS_LAYER_DOWNSAMPLE, CKKS_EINVAL, "unknown layer kind");
        CK_CHECK(L.n_in >= 1 && L.n_in <= 64 && L.n_out >= 1 && L.n_out <= 64, CKKS_EINVAL,
                 "a layer has 1 to 64 ciphertexts in and out");
        CK_CHECK(L.boot != nullptr, CKKS_EINVAL, "a layer needs its bootstrapping configuration");
        CK_CHECK(L.k >= 1 && L.k <= L.n_in, CKKS_EINVAL, "a layer's outputs read 1 to n_in inputs each");
        CK_CHECK(!L.in_index.empty() || L.k == L.n_in, CKKS_EINVAL, "without input indices every output reads all");
        CK_CHECK(L.in_index.empty() || (int)L.in_index.size() == L.n_out * L.k, CKKS_EINVAL,
                 "a layer needs n_out x k input indices");
        for (int i : L.in_index) CK_CHECK(i >= 0 && i < L.n_in, CKKS_EINVAL, "an input index is out of range");
        CK_CHECK((int)L.convs.size() == L.k * L.n_out, CKKS_EINVAL, "a layer needs n_out x k conv sets");
        for (const ckks_ptset* p : L.convs) CK_CHECK(p != nullptr, CKKS_EINVAL, "a conv set is NULL");
        if (k > 0) CK_CHECK(L.n_in == m.layers[k - 1].n_out, CKKS_EINVAL, "a layer's inputs are the previous outputs");
        if (L.kind == CKKS_LAYER_DOWNSAMPLE) {
            CK_CHECK(k > 0 && m.layers[k - 1].kind == CKKS_LAYER_BLOCK, CKKS_EINVAL,
                     "a downsampling layer follows a block layer (it takes that layer's EvalMod outputs)");
            CK_CHECK(L.boot_in != nullptr, CKKS_EINVAL, "a downsampling layer needs bt_in");
        }
    }
    m.n_in = m.layers.front().n_in;
    m.n_out = m.layers.back().n_out;
    m.in_level = m.layers.front().convs[0]->level;
    m.in_scale = c->delta[m.in_level];
    m.out_level = m.layers.back().boot->l_out;
    m.out_scale = c->delta[m.out_level];
    const size_t win = m.in_words(c->n), wout = m.out_words(c->n);
    // this model's staging buffers and graphs in every slot, kept until the server is destroyed
    // (the graphs refer to the buffers); they join the slots only once the whole model is
    // recorded, so that a failure leaves the slots' per-model vectors aligned with the models
    struct Staged {
        u64 *d_in = nullptr, *d_out = nullptr, *h_in = nullptr, *h_out = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<Staged> st(s->slots.size());
    auto release = [&] {
        for (Staged& x : st) {
            if (x.exec) cudaGraphExecDestroy(x.exec);
            if (x.graph) cudaGraphDestroy(x.graph);
            if (x.d_in) cudaFree(x.d_in);
            if (x.d_out) cudaFree(x.d_out);
            if (x.h_in) cudaFreeHost(x.h_in);
            if (x.h_out) cudaFreeHost(x.h_out);
        }
    };
    long long l0 = 0;
    try {
        for (Staged& x : st) {
            CUDA_CHECK(cudaMalloc((void**)&x.d_in, win * 8));
            CUDA_CHECK(cudaMalloc((void**)&x.d_out, wout * 8));
            CUDA_CHECK(cudaMallocHost((void**)&x.h_in, win * 8));
            CUDA_CHECK(cudaMallocHost((void**)&x.h_out, wout * 8));
            CUDA_CHECK(cudaMemset(x.d_in, 0, win * 8));
        }
        // one eager request: builds lazily created tables, checks keys and levels, and
        // measures the temporaries' peak in the context's memory pool
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        cudaMemPool_t pool;
        CUDA_CHECK(cudaDeviceGetDefaultMemPool(&pool, s->device));
        unsigned long long zero = 0, base = 0, high = 0;   // the pool attributes are 64-bit
        CUDA_CHECK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &base));
        CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
        l0 = c->launches;
        run_model(s, m, st[0].d_in, st[0].d_out);
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        m.kernels = c->launches - l0;
        CUDA_CHECK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
        m.footprint = high > base ? (long long)(high - base) : 0;
        if (s->sp.hbm_budget > 0)
            CK_CHECK(m.footprint <= s->sp.hbm_budget, CKKS_ENOMEM, "one request of this model exceeds the HBM budget");
        for (Staged& x : st) {
            CUDA_CHECK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            try {
                run_model(s, m, x.d_in, x.d_out);
            } catch (...) {
                cudaGraph_t tmp = nullptr;
                cudaStreamEndCapture(c->stream, &tmp);
                if (tmp) cudaGraphDestroy(tmp);
                throw;
            }
            CUDA_CHECK(cudaStreamEndCapture(c->stream, &x.graph));
            CUDA_CHECK(cudaGraphInstantiate(&x.exec, x.graph, 0));
        }
    } catch (...) {
        release();
        throw;
    }
    const int id = (int)s->models.size();
    for (size_t k = 0; k < s->slots.size(); ++k) {
        Slot& sl = s->slots[k];
        sl.d_in.push_back(st[k].d_in);
        sl.d_out.push_back(st[k].d_out);
        sl.h_in.push_back(st[k].h_in);
        sl.h_out.push_back(st[k].h_out);
        sl.graph.push_back(st[k].graph);
        sl.exec.push_back(st[k].exec);
    }
    c->launches = l0 + m.kernels;
    s->models.push_back(std::move(m));
    *model_id = id;
}

}  // namespace

extern "C" {

int ckks_server_add_model(ckks_server* s, int n_blocks, const ckks_ptset* const* convs, const ckks_boot* const* boots,
                          int* model_id) {
    if (!s) return CKKS_EINVAL;
    return sguard(s, [&] {
        REQ(convs);
        REQ(boots);
        REQ(model_id);
        CK_CHECK(n_blocks >= 1 && n_blocks <= 64, CKKS_EINVAL, "n_blocks must be in [1, 64]");
        Model m;
        for (int b = 0; b < n_blocks; ++b) {
            REQ(convs[b]);
            REQ(boots[b]);
            Layer L;
            L.convs.push_back(convs[b]);
            L.boot = boots[b];
            L.k = 1;
            m.layers.push_back(std::move(L));
        }
        add_model_impl(s, std::move(m), model_id);
    });
}

int ckks_server_add_model_layers(ckks_server* s, int n_layers, const ckks_server_layer* layers, int* model_id) {
    if (!s) return CKKS_EINVAL;
    return sguard(s, [&] {
        REQ(layers);
        REQ(model_id);
        CK_CHECK(n_layers >= 1 && n_layers <= 64, CKKS_EINVAL, "n_layers must be in [1, 64]");
        Model m;
        for (int k = 0; k < n_layers; ++k) {
            const ckks_server_layer& d = layers[k];
            CK_CHECK(d.n_in >= 1 && d.n_in <= 64 && d.n_out >= 1 && d.n_out <= 64, CKKS_EINVAL,
                     "a layer has 1 to 64 ciphertexts in and out");
            REQ(d.convs);
            CK_CHECK(d.k >= 1 && d.k <= d.n_in, CKKS_EINVAL, "a layer's outputs read 1 to n_in inputs each");
            Layer L;
            L.kind = d.kind;
            L.n_in = d.n_in;
            L.n_out = d.n_out;
            L.k = d.k;
            if (d.in_index) L.in_index.assign(d.in_index, d.in_index + (size_t)d.n_out * d.k);
            L.convs.assign(d.convs, d.convs + (size_t)d.k * d.n_out);
            L.boot = d.boot;
            L.boot_in = d.boot_in;
            m.layers.push_back(std::move(L));
        }
        add_model_impl(s, std::move(m), model_id);
    });
}

int ckks_server_model_shape(const ckks_server* s, int model_id, int* shape2) {
    if (!s || !shape2 || model_id < 0 || model_id >= (int)s->models.size()) return CKKS_EINVAL;
    shape2[0] = s->models[model_id].n_in;
    shape2[1] = s->models[model_id].n_out;
    return CKKS_OK;
}

int ckks_server_start(ckks_server* s) {
    if (!s) return CKKS_EINVAL;
    return sguard(s, [&] {
        CK_CHECK(!s->started, CKKS_EINVAL, "server already started");
        CK_CHECK(!s->models.empty(), CKKS_EINVAL, "no model");
        s->started = true;
        s->worker = std::thread(worker_main, s);
    });
}

int ckks_server_submit(ckks_server* s, int model_id, const uint64_t* host_in, int level, double scale,
                       uint64_t* request_id) {
    if (!s) return CKKS_EINVAL;
    return sguard(s, [&] {
        REQ(host_in);
        REQ(request_id);
        CK_CHECK(s->started, CKKS_EINVAL, "server not started");
        CK_CHECK(model_id >= 0 && model_id < (int)s->models.size(), CKKS_EINVAL, "unknown model");
        const Model& m = s->models[model_id];
        CK_CHECK(level == m.in_level, CKKS_EINVAL, "input level differs from the model's input level");
        CK_CHECK(scale == m.in_scale, CKKS_EINVAL, "input scale differs from the model's input scale");
        CK_CHECK(s->sp.hbm_budget == 0 || m.footprint <= s->sp.hbm_budget, CKKS_ENOMEM, "request exceeds the budget");
        Request r;
        r.model = model_id;
        r.in.assign(host_in, host_in + m.in_words(s->ctx->n));
        r.t_submit = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            r.id = s->next_id++;
            *request_id = r.id;
            s->queue.push_back(r.id);
            s->reqs.emplace(r.id, std::move(r));
        }
        s->cv.notify_all();
    });
}

int ckks_server_poll(ckks_server* s, uint64_t id, int* state) {
    if (!s || !state) return CKKS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return CKKS_EINVAL;
    *state = it->second.state;
    return CKKS_OK;
}

int ckks_server_wait(ckks_server* s, uint64_t id, double timeout_s, int* state) {
    if (!s || !state) return CKKS_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return CKKS_EINVAL;
    auto final_state = [&] {
        const int st = it->second.state;
        return st == CKKS_REQ_DONE || st == CKKS_REQ_FAILED || st == CKKS_REQ_CANCELLED;
    };
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s < 0 ? 0 : timeout_s), final_state);
    *state = it->second.state;
    return ok ? CKKS_OK : CKKS_ETIMEOUT;
}

int ckks_server_result(ckks_server* s, uint64_t id, uint64_t* host_out, int* level, double* scale) {
    if (!s) return CKKS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return CKKS_EINVAL;
    Request& r = it->second;
    if (r.state != CKKS_REQ_DONE) {
        s->err = r.state == CKKS_REQ_FAILED ? "request failed: " + r.err : "request not finished";
        return CKKS_EINVAL;
    }
    const Model& m = s->models[r.model];
    if (level) *level = m.out_level;
    if (scale) *scale = m.out_scale;
    if (host_out) {
        std::copy(r.out.begin(), r.out.end(), host_out);
        s->reqs.erase(it);
    }
    return CKKS_OK;
}

int ckks_server_cancel(ckks_server* s, uint64_t id) {
    if (!s) return CKKS_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return CKKS_EINVAL;
        it->second.cancel = true;
    }
    s->cv.notify_all();
    return CKKS_OK;
}

int ckks_server_stats(ckks_server* s, double* out) {
    if (!s || !out) return CKKS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out[0] = (double)s->completed;
    out[1] = (double)s->failed;
    out[2] = (double)s->cancelled;
    out[3] = percentile(s->lat_ms, 0.50);
    out[4] = percentile(s->lat_ms, 0.99);
    double sum = 0;
    for (double v : s->lat_ms) sum += v;
    out[5] = s->lat_ms.empty() ? 0.0 : sum / (double)s->lat_ms.size();
    out[6] = (double)s->max_in_flight;
    out[7] = (double)s->kernels;
    return CKKS_OK;
}

int ckks_server_reset_stats(ckks_server* s) {
    if (!s) return CKKS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->completed = s->failed = s->cancelled = s->kernels = 0;
    s->max_in_flight = s->in_flight;
    s->lat_ms.clear();
    return CKKS_OK;
}

int ckks_server_model_info(const ckks_server* s, int model_id, double* out) {
    if (!s || !out || model_id < 0 || model_id >= (int)s->models.size()) return CKKS_EINVAL;
    const Model& m = s->models[model_id];
    out[0] = m.in_level;
    out[1] = m.in_scale;
    out[2] = m.out_level;
    out[3] = m.out_scale;
    out[4] = (double)m.footprint;
    out[5] = (double)m.kernels;
    return CKKS_OK;
}

const char* ckks_server_last_error(const ckks_server* s) { return s ? s->err.c_str() : "null server"; }

int ckks_server_destroy(ckks_server* s) {
    delete s;
    return CKKS_OK;
}

}  // extern "C"
