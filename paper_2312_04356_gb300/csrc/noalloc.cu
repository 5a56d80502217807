// Rescale that allocates no device memory.
//
// Some callers cannot allocate device memory while they run: code recorded into a CUDA
// graph without the memory-pool nodes, real-time serving loops that forbid cudaMalloc
// because it can synchronise the device, or hosts that hand the library a fixed memory
// budget.  ckks_rescale_noalloc gives them the rescale of ckks_rescale with its scratch
// (the dropped limb in the coefficient domain and its centred lift into every other
// limb) taken from one file-scope device array instead of the stream-ordered pool.
#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace {

// 2^22 words = 32 MiB: the lift needs (2 level + 2) N words, i.e. levels up to 31 at N = 2^16.
constexpr size_t kScratchWords = (size_t)1 << 22;
__device__ __align__(256) u64 g_rescale_scratch[kScratchWords];

std::mutex g_scratch_mu;
std::unordered_map<int, u64*> g_scratch_addr;   // device ordinal -> device address of the array

// The array's name is only a host-side handle; the address a kernel may use is looked
// up once per device, with that device current.  The look-up is not allowed while `stream`
// is being captured into a CUDA graph: such a first call is refused with a clear error.
u64* scratch_for_current_device(cudaStream_t stream) {
    int dev = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    auto it = g_scratch_addr.find(dev);
    if (it != g_scratch_addr.end()) return it->second;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CUDA_CHECK(cudaStreamIsCapturing(stream, &cs));
    CK_CHECK(cs == cudaStreamCaptureStatusNone, CKKS_EINVAL,
             "ckks_rescale_noalloc: the first call on a device looks up the scratch array's address and "
             "cannot run inside a stream capture; call it once before capturing");
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rescale_scratch);
    if (e != cudaSuccess)
        CK_THROW(CKKS_ECUDA, std::string("cudaGetSymbolAddress(rescale scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = (u64*)p;
    return (u64*)p;
}

}  // namespace

extern "C" int ckks_rescale_noalloc(ckks_ctx* ctx, const uint64_t* d_in, int level, uint64_t* d_out) {
    if (!ctx) return CKKS_EINVAL;
    const bool timing = ctx->timing;
    ctx->timing = false;   // per-kernel timing would create CUDA events
    int rc = CKKS_OK;
    try {
        CK_CHECK(d_in && d_out, CKKS_EINVAL, "d_in / d_out is NULL");
        CK_CHECK(level >= 1 && level <= ctx->L, CKKS_EINVAL, "level must be in 1..L");
        const size_t n = ctx->n;
        const size_t need = (2 * (size_t)level + 2) * n;
        CK_CHECK(need <= kScratchWords, CKKS_EINVAL,
                 "ckks_rescale_noalloc: needs " + std::to_string(need) + " scratch words, the static array holds " +
                     std::to_string(kScratchWords) + " (lower the level or use ckks_rescale)");
        const size_t nl = (size_t)level + 1;
        const u64* in0 = reinterpret_cast<const u64*>(d_in);
        const u64* in1 = in0 + nl * n;
        u64* out0 = reinterpret_cast<u64*>(d_out);
        CK_CHECK(out0 + 2 * level * n <= in0 || in0 + 2 * nl * n <= out0, CKKS_EINVAL,
                 "d_out must not overlap d_in");
        u64* scratch = scratch_for_current_device(ctx->stream);
        u64* last = scratch;            // [2][N]: the dropped limb of c0 and c1
        u64* lift = scratch + 2 * n;    // [2][level][N]
        CUDA_CHECK(cudaMemcpyAsync(last, in0 + (size_t)level * n, n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        CUDA_CHECK(cudaMemcpyAsync(last + n, in1 + (size_t)level * n, n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        kern::ntt_inverse(ctx, last, 2, ctx->d_iota + level, 1);
        kern::lift_centred(ctx, last, level, lift, 2 * level, ctx->d_iota, level, n);   // both polynomials
        kern::ntt_forward(ctx, lift, 2 * level, ctx->d_iota, level);
        const u64* s = ctx->d_qlinv + (size_t)level * ctx->nq;
        const u64* sp = ctx->d_qlinv + (size_t)ctx->nq * ctx->nq + (size_t)level * ctx->nq;
        kern::sub_mul_scalar(ctx, in0, lift, s, sp, out0, 2 * level, ctx->d_iota, level, (size_t)nl * n);
        ctx->ops["rescale"]++;
    } catch (const CkksError& e) {
        ctx->err = e.msg;
        rc = e.code;
    }
    ctx->timing = timing;
    return rc;
}
