// Fused FP32 RK4 step with part of its on-chip state in tensor memory (TMEM).
//
// The z-marching tile of patch_tile.cuh keeps, per thread and column pair,
// register rings of the spin planes s and of the RK accumulator y = s + sum_j
// b_j dt K_j (Eq. LLL integrated by the Appendix's RK4 tableau).  Here the
// spin planes that are only read again one or two iterations later (stage
// 1's z-1 plane and stage 2's base s(t+2), stage 3's base s(t+1)) and the
// accumulators of the planes in flight live in the SM's tensor memory
// instead: each warp owns 64 columns of its 32-lane quarter (s slots at
// columns 0, 8, 16, 24 and y slots at 32 .. 56, six 32-bit words per slot =
// three float2 components of the thread's column pair).  A stage loads its y
// (and base) at its start and waits for them only where it adds its
// increment, so the load latency hides behind the stencil and the right-hand
// side.  The registers freed this way (128 per thread instead of 160) allow a
// 28-row tile of 448 threads: 20 output rows per tile, which on large
// lattices needs no z chunks at all.  The arithmetic of every site, and so
// every result, is bitwise that of the register-ring kernel.
//
// Used for RK4 steps without per-site fields, stage stores or a fused pulse.
// tcgen05.alloc takes 256 of the SM's 512 TMEM columns; the kernel's
// registers and shared memory leave room for one of its CTAs per SM, so its
// CTAs never compete for the columns (an allocation waits only while another
// kernel's CTA on the same SM holds more than 256 of them).
#pragma once
#include "patch_tile.cuh"

namespace spin {
namespace {

// the TMEM variant's tile: 16 x 28 threads, one row per thread
template <>
struct PatchShape<4, 3> {
    static constexpr int PY = 1, TY = 28;
};
constexpr int kTmemVariant = 3;
constexpr unsigned kTmemCols = 256;

// six 32-bit words (three float2) per thread from TMEM column ta on
__device__ __forceinline__ void tm_ld6(unsigned ta, unsigned (&r)[6]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(ta)
                 : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];\n" : "=r"(r[4]), "=r"(r[5]) : "r"(ta + 4) : "memory");
}
// wait for this thread's TMEM loads; the named registers are read only after
// it (they are operands of the wait, so no use is scheduled before it)
__device__ __forceinline__ void tm_wait_ld(unsigned (&r)[6]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5])::"memory");
}
__device__ __forceinline__ void tm_wait_ld(unsigned (&r)[6], unsigned (&q)[6]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(q[0]), "+r"(q[1]),
                   "+r"(q[2]), "+r"(q[3]), "+r"(q[4]), "+r"(q[5])::"memory");
}
__device__ __forceinline__ void tm_st6(unsigned ta, const f2 (&v)[3]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(ta),
                 "r"(__float_as_uint(v[0].x)), "r"(__float_as_uint(v[0].y)), "r"(__float_as_uint(v[1].x)),
                 "r"(__float_as_uint(v[1].y))
                 : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};\n" ::"r"(ta + 4), "r"(__float_as_uint(v[2].x)),
                 "r"(__float_as_uint(v[2].y))
                 : "memory");
}
// this thread's earlier TMEM stores are complete (before it loads them back)
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tm_f2(const unsigned (&r)[6], f2 (&v)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = make_float2(__uint_as_float(r[2 * c]), __uint_as_float(r[2 * c + 1]));
}
__device__ __forceinline__ unsigned tm_s(unsigned tw, int slot) { return tw + 8u * (unsigned)slot; }
__device__ __forceinline__ unsigned tm_y(unsigned tw, int slot) { return tw + 32u + 8u * (unsigned)slot; }

// One wavefront iteration: stage j on plane t+4-j (slot (P+4-j) & 3).  In
// registers: sc = s(t+3) (stage 1's centre plane, fetched the iteration
// before), the new plane s(t+4), and the X_2..X_4 rings; in TMEM: s(t+2),
// s(t+1) and y of planes t .. t+3.
template <bool PREC, int P>
__device__ __forceinline__ void tm_iteration(const PatchArgs& a, f2 (&xr)[3][4][3], f2 (&sc)[3], float* __restrict__ sh,
                                             float* __restrict__ stg, PThread<1>& th, int i, int t0, int z0, int tid,
                                             unsigned tw) {
    constexpr int S = 4, V = kTmemVariant, ROWS = PatchShape<4, V>::TY, TILE = ROWS * kRS;
    float* shb = sh + (P & 1) * (S * 3 * TILE);
    const int cy0 = th.ty, cx0 = 2 * th.tx;
    // 1. publish the stage inputs for the y-neighbours
#pragma unroll
    for (int j = 1; j <= S; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const f2 v = (j == 1) ? sc[c] : xr[j - 2][(P + S - j) & 3][c];
            *reinterpret_cast<f2*>(shb + ((j - 1) * 3 + c) * TILE + cy0 * kRS + cx0) = v;
        }
    // 2. plane t+4 from the staging ring, plane t+6 requested
    const int t = i + t0;
    issue_plane<S, V>(a, stg, th, (P + S + 2) & 3, th.gz_issue, tid);
    th.gz_issue = th.gz_issue + 1 == a.nz ? 0 : th.gz_issue + 1;
    cp_async_wait<2>();
    f2 snew[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) snew[c] = *reinterpret_cast<const f2*>(stage_pair<S, V>(stg, (P + S) & 3, c, 0, tid));
    if (a.bc) {
        const float zin = (t + S >= 0 && t + S < a.nz) ? 1.f : 0.f;
        const f2 m = make_float2(th.cmask[0].x * zin, th.cmask[0].y * zin);
#pragma unroll
        for (int c = 0; c < 3; ++c) snew[c] = mul2(snew[c], m);
    }
    tm_wait_st();   // the previous iteration's TMEM stores are complete
    unsigned rs2[6];
    tm_ld6(tm_s(tw, (P + 2) & 3), rs2);   // s(t+2)
    __syncthreads();

    // 3. stages 1..4
    const int up = cy0 > 0 ? cy0 - 1 : cy0;
    const int dn = cy0 + 1 < ROWS ? cy0 + 1 : cy0;
    f2 nb_up[3], nb_dn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        nb_up[c] = *reinterpret_cast<const f2*>(shb + c * TILE + up * kRS + cx0);
        nb_dn[c] = *reinterpret_cast<const f2*>(shb + c * TILE + dn * kRS + cx0);
    }
    tm_wait_ld(rs2);
    f2 s2[3];
    tm_f2(rs2, s2);
#pragma unroll
    for (int j = 1; j <= S; ++j) {
        // warp-uniform activity, as in the register-ring kernel
        const bool active = (2 * th.warp_row + 1 >= j) && (2 * th.warp_row < ROWS - j) && (i >= 2 * j - 2);
        const int slot = (P + S - j) & 3;
        const int sm = (slot + 3) & 3, sp = (slot + 1) & 3;
        if (active) {
            unsigned ry[6], rb[6];
            if (j >= 2) tm_ld6(tm_y(tw, slot), ry);
            if (j == 3) tm_ld6(tm_s(tw, slot), rb);
            f2 C[3], sum[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                C[c] = (j == 1) ? sc[c] : xr[j - 2][slot][c];
                const f2 ZM = (j == 1) ? s2[c] : xr[j - 2][sm][c];
                const f2 ZP = (j == 1) ? snew[c] : xr[j - 2][sp][c];
                const float L = __shfl_up_sync(0xffffffffu, C[c].y, 1, kPT);
                const float Rr = __shfl_down_sync(0xffffffffu, C[c].x, 1, kPT);
                const f2 xs = make_float2(__fadd_rn(L, C[c].y), __fadd_rn(C[c].x, Rr));
                sum[c] = add2(add2(add2(xs, add2(nb_up[c], nb_dn[c])), ZM), ZP);
            }
            if (j < S) {
                const float* shn = shb + j * 3 * TILE;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    nb_up[c] = *reinterpret_cast<const f2*>(shn + c * TILE + up * kRS + cx0);
                    nb_dn[c] = *reinterpret_cast<const f2*>(shn + c * TILE + dn * kRS + cx0);
                }
            }
            f2 f[3];
            rhs_pair<PREC>(sum, C, a.J, a.twoD, a.Hx, a.Hy, a.Hz, a.lambda, f);
            f2 y[3], base[3];
            if (j == 1) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    base[c] = sc[c];
                    y[c] = fma2(sp2(a.bdt[0]), f[c], sc[c]);
                }
            } else {
                if (j == 3) {
                    tm_wait_ld(ry, rb);
                    tm_f2(rb, base);
                } else {
                    tm_wait_ld(ry);
                    if (j == 2) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) base[c] = s2[c];
                    }
                }
                f2 yo[3];
                tm_f2(ry, yo);
#pragma unroll
                for (int c = 0; c < 3; ++c) y[c] = fma2(sp2(a.bdt[j - 1]), f[c], yo[c]);
            }
            if (j < S) {
#pragma unroll
                for (int c = 0; c < 3; ++c) xr[j - 1][slot][c] = fma2(sp2(a.cdt[j - 1]), f[c], base[c]);
                tm_st6(tm_y(tw, slot), y);
            } else if (t >= z0 && t < z0 + a.tz && t < a.nz) {
                // finished plane t: renormalise and store
                const int b = t * th.plane;
                f2 ox = y[0], oy = y[1], oz = y[2];
                if (a.renorm) {
                    const f2 n2 = fma2(ox, ox, fma2(oy, oy, mul2(oz, oz)));
                    const f2 inv = make_float2(rsqrtf(n2.x), rsqrtf(n2.y));
                    ox = mul2(ox, inv);
                    oy = mul2(oy, inv);
                    oz = mul2(oz, inv);
                }
                if (a.pair8out) {
                    if (th.out[0][0]) {
                        const int site = b + th.col[0][0];
                        *reinterpret_cast<f2*>(a.out0 + site) = ox;
                        *reinterpret_cast<f2*>(a.out1 + site) = oy;
                        *reinterpret_cast<f2*>(a.out2 + site) = oz;
                    }
                } else {
                    const float vx[2] = {ox.x, ox.y}, vy[2] = {oy.x, oy.y}, vz[2] = {oz.x, oz.y};
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if (!th.out[0][e]) continue;
                        const int site = b + th.col[0][e];
                        a.out0[site] = vx[e];
                        a.out1[site] = vy[e];
                        a.out2[site] = vz[e];
                    }
                }
            }
        }
    }
    tm_st6(tm_s(tw, (P + 3) & 3), sc);   // s(t+3) leaves the registers for TMEM
#pragma unroll
    for (int c = 0; c < 3; ++c) sc[c] = snew[c];
}

// One CTA's tile (bx, by) and z chunk bz; tm_slot is a shared word that
// receives the TMEM base address.
template <bool PREC>
__device__ __forceinline__ void tm_tile(const PatchArgs& a, int bx, int by, int bz, float* __restrict__ sh,
                                        unsigned* tm_slot) {
    constexpr int S = 4, V = kTmemVariant, ROWS = PatchShape<4, V>::TY;
    float* stg = sh + 2 * S * 3 * ROWS * kRS;
    const int tid = threadIdx.y * kPT + threadIdx.x;
    PThread<1> th;
    th.tx = threadIdx.x;
    th.ty = threadIdx.y;
    th.bad = false;
    th.stg_off[0] = 0;
    th.warp_row = __shfl_sync(0xffffffffu, (int)((threadIdx.y * kPT + threadIdx.x) >> 5), 0);
    constexpr int OUTX = kPC - 2 * S, OUTY = ROWS - 2 * S;
    th.plane = a.nx * a.ny;
    {
        const int cy = th.ty;
        const int gyu = by * OUTY - S + cy;
        const int gy = wrapi(gyu, a.ny);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int cx = 2 * th.tx + e;
            const int gxu = bx * OUTX - S + cx;
            th.col[0][e] = gy * a.nx + wrapi(gxu, a.nx);
            th.out[0][e] = cx >= S && cx < kPC - S && cy >= S && cy < ROWS - S && gxu < a.nx && gyu < a.ny;
            const float in = (gxu >= 0 && gxu < a.nx && gyu >= 0 && gyu < a.ny) ? 1.f : 0.f;
            if (e == 0) th.cmask[0].x = a.bc ? in : 1.f;
            else th.cmask[0].y = a.bc ? in : 1.f;
        }
    }
    // tensor memory: warp w uses lanes 32 (w % 4) .. +31 (its quarter) and
    // the 64 columns from 64 (w / 4), so 256 columns serve up to 16 warps
    static_assert(kPT * PatchShape<4, V>::TY / 32 <= 16, "TMEM columns per warp quarter");
    if (th.warp_row == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tm_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tbase = *tm_slot;
    const unsigned tw = tbase + ((unsigned)(32 * (th.warp_row & 3)) << 16) + 64u * (unsigned)(th.warp_row >> 2);

    const int z0 = bz * a.tz;
    const int t0 = z0 - 2 * S + 2;
    f2 xr[3][4][3], sc[3];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < 3; ++j) xr[j][q][c] = make_float2(0.f, 0.f);
    {
        // planes t0+2 (to TMEM slot 2) and t0+3 (sc) straight from global memory
        f2 s2[3];
        const int b2 = wrapi(t0 + 2, a.nz) * th.plane, b3 = wrapi(t0 + 3, a.nz) * th.plane;
        const int o0 = th.col[0][0], o1 = th.col[0][1];
        s2[0] = make_float2(__ldg(a.in0 + b2 + o0), __ldg(a.in0 + b2 + o1));
        s2[1] = make_float2(__ldg(a.in1 + b2 + o0), __ldg(a.in1 + b2 + o1));
        s2[2] = make_float2(__ldg(a.in2 + b2 + o0), __ldg(a.in2 + b2 + o1));
        sc[0] = make_float2(__ldg(a.in0 + b3 + o0), __ldg(a.in0 + b3 + o1));
        sc[1] = make_float2(__ldg(a.in1 + b3 + o0), __ldg(a.in1 + b3 + o1));
        sc[2] = make_float2(__ldg(a.in2 + b3 + o0), __ldg(a.in2 + b3 + o1));
        if (a.bc) {
            const float z2 = (t0 + 2 >= 0 && t0 + 2 < a.nz) ? 1.f : 0.f;
            const float z3 = (t0 + 3 >= 0 && t0 + 3 < a.nz) ? 1.f : 0.f;
            const f2 m2 = make_float2(th.cmask[0].x * z2, th.cmask[0].y * z2);
            const f2 m3 = make_float2(th.cmask[0].x * z3, th.cmask[0].y * z3);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                s2[c] = mul2(s2[c], m2);
                sc[c] = mul2(sc[c], m3);
            }
        }
        tm_st6(tm_s(tw, 2), s2);
    }
    issue_plane<S, V>(a, stg, th, S & 3, wrapi(t0 + S, a.nz), tid);
    issue_plane<S, V>(a, stg, th, (S + 1) & 3, wrapi(t0 + S + 1, a.nz), tid);
    th.gz_issue = wrapi(t0 + S + 2, a.nz);
    int i = 0;
    for (; i + 4 <= a.n_iter; i += 4) {
        tm_iteration<PREC, 0>(a, xr, sc, sh, stg, th, i + 0, t0, z0, tid, tw);
        tm_iteration<PREC, 1>(a, xr, sc, sh, stg, th, i + 1, t0, z0, tid, tw);
        tm_iteration<PREC, 2>(a, xr, sc, sh, stg, th, i + 2, t0, z0, tid, tw);
        tm_iteration<PREC, 3>(a, xr, sc, sh, stg, th, i + 3, t0, z0, tid, tw);
    }
    if (i < a.n_iter) tm_iteration<PREC, 0>(a, xr, sc, sh, stg, th, i + 0, t0, z0, tid, tw);
    if (i + 1 < a.n_iter) tm_iteration<PREC, 1>(a, xr, sc, sh, stg, th, i + 1, t0, z0, tid, tw);
    if (i + 2 < a.n_iter) tm_iteration<PREC, 2>(a, xr, sc, sh, stg, th, i + 2, t0, z0, tid, tw);
    cp_async_wait<0>();   // no copy may land in shared memory after the tile is done
    // every warp's TMEM accesses are complete before the columns are freed
    tm_wait_st();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (th.warp_row == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(kTmemCols) : "memory");
    }
}

}  // namespace
}  // namespace spin
