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

struct Model {
    std::vector<const ckks_ptset*> convs;
    std::vector<const ckks_boot*> boots;
    int in_level = 0, out_level = 0;
    double in_scale = 0, out_scale = 0;
    long long footprint = 0;      // peak bytes of temporaries of one request
    long long kernels = 0;        // kernel launches of one request's graph
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
    u64* d_in = nullptr;          // coefficient-domain input limbs
    u64* d_out = nullptr;         // coefficient-domain output limbs
    u64* h_in = nullptr;          // pinned staging
    u64* h_out = nullptr;
    size_t in_words = 0, out_words = 0;
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

// One request of model m, reading d_in and writing d_out (both coefficient domain).
void run_model(ckks_server* s, const Model& m, const u64* d_in, u64* d_out) {
    ckks_ctx* c = s->ctx;
    ckks_ct x = ops::new_ct(c, m.in_level, m.in_scale);
    const size_t win = 2 * (size_t)(m.in_level + 1) * c->n;
    CUDA_CHECK(cudaMemcpyAsync(x.buf.ptr, d_in, win * 8, cudaMemcpyDeviceToDevice, c->stream));
    kern::ntt_forward(c, x.buf.ptr, 2 * (m.in_level + 1), c->d_iota, m.in_level + 1);
    for (size_t b = 0; b < m.convs.size(); ++b) {
        if (x.level != m.convs[b]->level) x = ops::level_down(x, m.convs[b]->level);
        x = ops::block(*s->keys, *m.boots[b], *m.convs[b], x);
    }
    CK_CHECK(x.level == m.out_level, CKKS_EINVAL, "model output level changed");
    const size_t wout = 2 * (size_t)(x.level + 1) * c->n;
    CUDA_CHECK(cudaMemcpyAsync(d_out, x.buf.ptr, wout * 8, cudaMemcpyDeviceToDevice, c->stream));
    kern::ntt_inverse(c, d_out, 2 * (x.level + 1), c->d_iota, x.level + 1);
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
            r.out.assign(sl.h_out, sl.h_out + 2 * (size_t)(s->models[r.model].out_level + 1) * s->ctx->n);
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
        std::copy(r.in.begin(), r.in.end(), sl.h_in);
        cudaError_t e = cudaMemcpyAsync(sl.d_in, sl.h_in, r.in.size() * 8, cudaMemcpyHostToDevice, sl.stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec[r.model], sl.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.h_out, sl.d_out, 2 * (size_t)(m.out_level + 1) * s->ctx->n * 8,
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
        if (sl.d_in) cudaFree(sl.d_in);
        if (sl.d_out) cudaFree(sl.d_out);
        if (sl.h_in) cudaFreeHost(sl.h_in);
        if (sl.h_out) cudaFreeHost(sl.h_out);
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

int ckks_server_add_model(ckks_server* s, int n_blocks, const ckks_ptset* const* convs, const ckks_boot* const* boots,
                          int* model_id) {
    if (!s) return CKKS_EINVAL;
    return sguard(s, [&] {
        REQ(convs);
        REQ(boots);
        REQ(model_id);
        CK_CHECK(!s->started, CKKS_EINVAL, "models are added before ckks_server_start");
        CK_CHECK(n_blocks >= 1 && n_blocks <= 64, CKKS_EINVAL, "n_blocks must be in [1, 64]");
        CK_CHECK(!s->ctx->timing, CKKS_EINVAL, "switch kernel timing off before recording graphs");
        ckks_ctx* c = s->ctx;
        Model m;
        for (int b = 0; b < n_blocks; ++b) {
            REQ(convs[b]);
            REQ(boots[b]);
            m.convs.push_back(convs[b]);
            m.boots.push_back(boots[b]);
        }
        m.in_level = convs[0]->level;
        m.in_scale = c->delta[m.in_level];
        m.out_level = boots[n_blocks - 1]->l_out;
        m.out_scale = c->delta[m.out_level];
        const size_t win = 2 * (size_t)(m.in_level + 1) * c->n, wout = 2 * (size_t)(m.out_level + 1) * c->n;
        // slot buffers sized for every model
        for (Slot& sl : s->slots) {
            if (sl.in_words < win) {
                if (sl.d_in) cudaFree(sl.d_in);
                if (sl.h_in) cudaFreeHost(sl.h_in);
                sl.d_in = nullptr;
                sl.h_in = nullptr;
                CUDA_CHECK(cudaMalloc((void**)&sl.d_in, win * 8));
                CUDA_CHECK(cudaMallocHost((void**)&sl.h_in, win * 8));
                CUDA_CHECK(cudaMemset(sl.d_in, 0, win * 8));
                sl.in_words = win;
            }
            if (sl.out_words < wout) {
                if (sl.d_out) cudaFree(sl.d_out);
                if (sl.h_out) cudaFreeHost(sl.h_out);
                sl.d_out = nullptr;
                sl.h_out = nullptr;
                CUDA_CHECK(cudaMalloc((void**)&sl.d_out, wout * 8));
                CUDA_CHECK(cudaMallocHost((void**)&sl.h_out, wout * 8));
                sl.out_words = wout;
            }
        }
        // one eager request: builds lazily created tables, checks keys and levels, and
        // measures the temporaries' peak in the context's memory pool
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        cudaMemPool_t pool;
        CUDA_CHECK(cudaDeviceGetDefaultMemPool(&pool, s->device));
        unsigned long long zero = 0, base = 0, high = 0;   // the pool attributes are 64-bit
        CUDA_CHECK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &base));
        CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
        const long long l0 = c->launches;
        run_model(s, m, s->slots[0].d_in, s->slots[0].d_out);
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        m.kernels = c->launches - l0;
        CUDA_CHECK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
        m.footprint = high > base ? (long long)(high - base) : 0;
        if (s->sp.hbm_budget > 0)
            CK_CHECK(m.footprint <= s->sp.hbm_budget, CKKS_ENOMEM, "one request of this model exceeds the HBM budget");
        const int id = (int)s->models.size();
        for (Slot& sl : s->slots) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t e = nullptr;
            CUDA_CHECK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            try {
                run_model(s, m, sl.d_in, sl.d_out);
            } catch (...) {
                cudaGraph_t tmp = nullptr;
                cudaStreamEndCapture(c->stream, &tmp);
                if (tmp) cudaGraphDestroy(tmp);
                throw;
            }
            CUDA_CHECK(cudaStreamEndCapture(c->stream, &g));
            const cudaError_t ie = cudaGraphInstantiate(&e, g, 0);
            if (ie != cudaSuccess) {
                cudaGraphDestroy(g);
                CUDA_CHECK(ie);
            }
            sl.graph.push_back(g);
            sl.exec.push_back(e);
        }
        c->launches = l0 + m.kernels;
        s->models.push_back(std::move(m));
        *model_id = id;
    });
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
        r.in.assign(host_in, host_in + 2 * (size_t)(level + 1) * s->ctx->n);
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
