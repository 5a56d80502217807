// Launch helpers and device routines shared by the kernel translation units.
#pragma once
#include "internal.h"

#include <atomic>

// ------------------------------------------------- dependent launches ----
// Every kernel of the library begins with griddep_entry(): it waits until the grids it depends
// on have completed and their writes are visible (griddepcontrol.wait; a no-op for a plain
// launch).  With that wait ahead of every memory access, a launch with programmatic stream
// serialization keeps stream order while the next grid is set up as the previous one
// drains, which hides most of the launch latency of eager calls.  Inside a CUDA graph
// capture the launches stay plain: a graph already removes that latency, and programmatic
// edges measured slightly slower there.
__device__ __forceinline__ void griddep_entry() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Opt a kernel in to more than 48 KB of dynamic shared memory, once per device (bit d of
// `done` records device d; concurrent first calls only repeat the same setting).
static inline void allow_dynamic_smem(const void* func, int bytes, std::atomic<unsigned>& done) {
    int dev = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    const unsigned bit = 1u << (dev & 31);
    if (done.load() & bit) return;
    CUDA_CHECK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done.fetch_or(bit);
}

template <typename... P, typename... A>
static inline void klaunch(const ckks_ctx* c, void (*k)(P...), dim3 grid, dim3 block, size_t smem, A... args) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (c->pdl) cudaStreamIsCapturing(c->stream, &cs);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = (c->pdl && cs == cudaStreamCaptureStatusNone) ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

// (hi:lo) mod q for any 128-bit value: hi (2^64 mod q) + lo mod q, canonical; lo is reduced
// as the Shoup product lo * 1 (companion floor(2^64 / q)), one high product instead of Barrett's
__device__ __forceinline__ u64 reduce128_lazy(u64 hi, u64 lo, const DevPrime& P) {
    const u64 q = P.m.q;
    u64 l = lo - __umul64hi(lo, P.inv64) * q;      // [0, 2q)
    if (l >= q) l -= q;
    return add_mod(mul_shoup(hi, P.r64, P.r64p, q), l, q);
}

// The rounding term of an exact base conversion, v = round(sum_i xh_i / q_i) (xh_i < q_i, at
// most 16 terms), in fixed point with 58 fractional bits: with 1/q_i = M_i 2^-(64 + b_i)
// (M_i = floor(2^(64 + b_i) / q_i), b_i = bitlen(q_i) - 1), term i is the 128-bit product
// xh_i M_i shifted right by sh_i = b_i + 6.  Each term is truncated by less than 2^-57 and the
// sum (< 16) by less than 2^-53 in all, against ~2^-49 for the same sum in FP64; the sum is
// never exactly a half-integer (Q is odd), so round-half-up is round-to-nearest.
__device__ __forceinline__ u64 conv_round_term(u64 xh, u64 m, int sh) {
    const u64 lo = xh * m, hi = __umul64hi(xh, m);
    return sh >= 64 ? hi >> (sh - 64) : (hi << (64 - sh)) | (lo >> sh);
}
__device__ __forceinline__ u64 conv_round_finish(u64 s) { return (s + (1ull << 57)) >> 58; }
