// Device helpers shared by the fused z-marching step kernels (chain
// tableaus and the two-segment six-stage step): the CTA column geometry, packed
// f32x2 arithmetic, cp.async staging and periodic index wrapping.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace spin {
namespace {

constexpr int kPT = 16;        // threads along x
constexpr int kPC = 2 * kPT;   // columns along x (two per thread, one float2)
constexpr int kRS = kPC;       // shared row stride (floats)

// A column pair (2m, 2m+1) is contiguous in a row of even length and never
// straddles the periodic wrap; with 8-byte aligned component arrays it can be
// fetched as one 8-byte copy.
__host__ __device__ __forceinline__ bool pairs_aligned(int nx, const float* p0, const float* p1, const float* p2) {
    return (nx & 1) == 0 && ((reinterpret_cast<unsigned long long>(p0) | reinterpret_cast<unsigned long long>(p1) |
                              reinterpret_cast<unsigned long long>(p2)) & 7ULL) == 0;
}

typedef float2 f2;
#ifndef SPIN_NO_F32X2
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
#else
// scalar FP32 per component (tuning comparison)
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y)); }
#endif
__device__ __forceinline__ f2 sp2(float v) { return make_float2(v, v); }

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(float* smem, const float* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const float* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---- mbarriers and bulk (TMA engine) copies between global and shared memory

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
// make initialised mbarriers visible to the other threads and to the async proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}
// try_wait with a suspend-time hint (ns): an unfinished phase suspends the
// warp instead of polling
constexpr unsigned kSuspendNs = 100000;
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity, giving up after a bounded number of
// suspended polls (a few seconds at most): then bit 0 of *err is set, *bad
// makes the thread skip its later waits, and the step's results are invalid
// (the host reports SPIN_ETIMEOUT).
constexpr int kWaitPolls = 1 << 15;
__device__ __forceinline__ void mbar_wait(unsigned long long* b, unsigned parity, int* err, bool& bad) {
    if (bad) return;
    for (int n = 0; n < kWaitPolls; ++n)
        if (mbar_try_wait(b, parity)) return;
    bad = true;
    if (err) atomicOr(err, 1);
}
// global -> shared, completion counted in bytes on an mbarrier (16-byte
// aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(smem)),
        "l"(gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// shared -> global, tracked in the issuing thread's bulk groups
__device__ __forceinline__ void bulk_s2g(void* gmem, const void* smem, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gmem), "r"(smem_addr(smem)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// at most N of this thread's bulk groups may still be reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
// at most N of this thread's bulk groups may still be incomplete
template <int N>
__device__ __forceinline__ void bulk_wait() {
    asm volatile("cp.async.bulk.wait_group %0;\n" ::"n"(N) : "memory");
}
// order this thread's generic shared-memory writes before later async-proxy reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ int wrapi(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// Right-hand side of Eq. (LLL) for a column pair: H = J sum_nn + H_ext
// (+ 2D s_z z), a = s x H, b = s x a, f = a - lambda b (precessional) or
// f = -lambda b (the slow equation, precession dropped).
template <bool PREC>
__device__ __forceinline__ void rhs_pair(const f2 (&sum)[3], const f2 (&cen)[3], float J, float twoD, float Hx,
                                         float Hy, float Hz, float lambda, f2 (&f)[3]) {
    const f2 hx = fma2(sp2(J), sum[0], sp2(Hx));
    const f2 hy = fma2(sp2(J), sum[1], sp2(Hy));
    f2 hz = fma2(sp2(J), sum[2], sp2(Hz));
    const f2 sx = cen[0], sy = cen[1], sz = cen[2];
    hz = fma2(sp2(twoD), sz, hz);
    const f2 nx_ = make_float2(-sx.x, -sx.y), ny_ = make_float2(-sy.x, -sy.y), nz_ = make_float2(-sz.x, -sz.y);
    const f2 ax = fma2(nz_, hy, mul2(sy, hz));
    const f2 ay = fma2(nx_, hz, mul2(sz, hx));
    const f2 az = fma2(ny_, hx, mul2(sx, hy));
    const f2 bx = fma2(nz_, ay, mul2(sy, az));
    const f2 by = fma2(nx_, az, mul2(sz, ax));
    const f2 bz = fma2(ny_, ax, mul2(sx, ay));
    if (PREC) {
        f[0] = fma2(sp2(-lambda), bx, ax);
        f[1] = fma2(sp2(-lambda), by, ay);
        f[2] = fma2(sp2(-lambda), bz, az);
    } else {
        f[0] = mul2(sp2(-lambda), bx);
        f[1] = mul2(sp2(-lambda), by);
        f[2] = mul2(sp2(-lambda), bz);
    }
}

}  // namespace
}  // namespace spin
