// Fused FP32 step for Butcher's six-stage fifth-order Runge-Kutta method
// (Appendix), as two z-marching segments of three stages each.
//
// Stage j of this tableau reads K_l = dt f(X_l) of every earlier stage at its
// own site, so one kernel over all six stages would need a tile halo of 6 and
// register rings for five stage inputs plus the K_l still to be combined.
// Cut after stage 3, what the last three stages need of the first three is
// four vectors per site (f_l = f(X_l); the tableau's a41 = a52 = a53 = b2 = 0):
//   X4 = s + dt (a42 f2 + a43 f3)
//   P5 = s + dt a51 f1                          X5 = P5 + dt a54 f4
//   P6 = s + dt (a61 f1 + a62 f2 + a63 f3)      X6 = P6 + dt (a64 f4 + a65 f5)
//   Py = s + dt (b1 f1 + b3 f3)                 y  = Py + dt (b4 f4 + b5 f5 + b6 f6)
// Segment A evaluates stages 1-3 from the state and writes (X4, P5, P6, Py);
// segment B evaluates stages 4-6 from them, renormalises and writes the new
// state.  Each segment is the chain step's wavefront with three stages: a
// 32-column x TY-row tile with a halo of 3 rows, marching along z, stage j on
// plane t+3-j at iteration t, x-neighbours by shuffles, y-neighbours through
// shared memory, z-neighbours from register rings indexed by plane & 3.
//
// The four carried vectors are one 48-byte record per site (X4 xyz, P5 xyz,
// P6 xyz, Py xyz), so a tile row of them is one contiguous run of global
// memory.  They move by bulk copies of the TMA engine, off the threads'
// load/store path: A assembles each plane's output records in shared memory
// and one lane per row stores the row (24 records) with one bulk copy; in B
// one lane per row fetches the row's 32 records (one or two runs where the
// row wraps around x) into a 4-slot ring, counted on the slot's mbarrier.
// Along x the tile needs a halo of 3 columns, like along y; its first column
// sits 4 columns left of the output window, at an even column, so that with
// rows of even length every thread's column pair is one aligned 8-byte word
// of the state arrays, and its output window is the 26 columns from tile
// column 3 (tile bx outputs global columns 26 bx - 1 .. 26 bx + 24, clipped to
// the lattice).  HBM traffic per site and step: 12 + 48 bytes for A, 48 + 12
// for B.
#include <cuda_runtime.h>

#include <algorithm>

#include "patch_common.cuh"
#include "spin_device.cuh"
#include "spin_internal.h"

namespace spin {

namespace {

constexpr int kH = 3;    // stages per segment = tile halo along x and y
constexpr int kHX = 4;   // tile origin: 4 columns left of the output window's first column - 1 (even: aligned pairs)
#ifndef SPIN_RK5_TY
#define SPIN_RK5_TY 20
#endif
constexpr int kTY = SPIN_RK5_TY;   // thread rows = tile rows (one row per thread)
constexpr int kNT = kPT * kTY;
constexpr int kOutX = kPC - 2 * kH, kOutY = kTY - 2 * kH;   // output window: tile columns [kH, kH + kOutX)
constexpr int kRec = 12;           // floats per site record of the carried vectors
constexpr int kRowBytes = kPC * kRec * 4;              // one tile row of records
constexpr int kSlotBytes = kTY * kRowBytes;            // one plane of the tile (B's ring slot)
constexpr int kOutBufFloats = kOutY * kOutX * kRec;    // A's output records of one plane

struct Rk5Args {
    const float* __restrict__ in0;   // A: the state s
    const float* __restrict__ in1;
    const float* __restrict__ in2;
    float* __restrict__ out0;        // B: the new state
    float* __restrict__ out1;
    float* __restrict__ out2;
    float* car;                      // per-site records (X4, P5, P6, Py): A writes, B reads
    int nx, ny, nz, tz, n_iter;
    float J, twoD, Hx, Hy, Hz, lambda;
    // dt x the nonzero Butcher coefficients of the Appendix's RK5
    float a21, a31, a32, a42, a43, a51, a54, a61, a62, a63, a64, a65;
    float b1, b3, b4, b5, b6;
    int renorm;
    int bc;                          // 1: free boundaries
    int pair8;                       // 1: column pairs are aligned 8-byte words of the state arrays
    int* err;                        // device status word: bit 0 set when a bounded wait gave up
};

struct R5Thread {
    int tx, ty, warp_row;
    int col[2];      // global column index gy*nx+gx of the pair's two sites
    bool out[2];
    int plane;       // nx*ny
    int gz_issue;    // wrapped z of the next plane to prefetch (t+5)
    f2 cmask;        // 1 for lattice columns, 0 outside a free-boundary lattice
    int grow;        // wrapped global y of the thread's row
    int gx0;         // wrapped global x of the tile's first column
    bool bad;        // a bounded wait of this thread gave up
};

// Register rings, slot = plane & 3.  x[j-1]: input of the segment's stage j
// (A: s, X2, X3; B: X4, X5, X6).  A keeps f1 (u) and f2 (v) until stage 3
// combines them; B keeps the partial X6 (u) and the partial y (v).
struct R5Rings {
    f2 x[3][4][3];
    f2 u[4][3];
    f2 v[4][3];
};

// A's staging ring of state planes fetched two iterations ahead with
// cp.async, 4 slots, thread-minor (a thread only reads back what it copied):
// 3 components x one column pair (8 bytes).
__device__ __forceinline__ float* r5_stage_a(float* stg, int slot, int c, int tid) {
    return stg + 2 * (((slot * 3 + c) * kNT) + tid);
}
// B's ring slot: the tile's rows of site records as laid out in global
// memory; the thread's column pair is 6 consecutive 16-byte words
__device__ __forceinline__ const float4* r5_slot_b(const unsigned char* slots, int slot, const R5Thread& th) {
    return reinterpret_cast<const float4*>(slots + slot * kSlotBytes + th.ty * kRowBytes + th.tx * 2 * kRec * 4);
}

// B: lane 0 of every row fetches that row's 32 records of (wrapped) plane gz
// into the slot, in contiguous runs (a run ends where the row wraps around x;
// at most ceil(32/nx)+1 runs), and counts their bytes on the slot's mbarrier.
__device__ __forceinline__ void r5_fetch_rows(const Rk5Args& a, unsigned char* slots, unsigned long long* bars,
                                              const R5Thread& th, int slot, int gz) {
    if (th.tx != 0) return;
    unsigned long long* bar = bars + slot;
    mbar_arrive_expect_tx(bar, kRowBytes);
    const int rowbase = gz * th.plane + th.grow * a.nx;
    unsigned char* dst = slots + slot * kSlotBytes + th.ty * kRowBytes;
    int x = th.gx0, done = 0;
    while (done < kPC) {
        const int n = min(kPC - done, a.nx - x);
        bulk_g2s(dst + done * kRec * 4, a.car + (size_t)kRec * (unsigned)(rowbase + x), (unsigned)(n * kRec * 4), bar);
        done += n;
        x = 0;
    }
}

// B: phase of slot (p & 3) that carries local plane p (planes 2, 3, 4, ...
// are fetched; slots 0 and 1 are first used by planes 4 and 5)
__device__ __forceinline__ unsigned r5_parity(int p) { return (unsigned)((p >> 2) - ((p & 3) < 2 ? 1 : 0)) & 1u; }

template <int SEG>
__device__ __forceinline__ void r5_issue(const Rk5Args& a, float* stg, const R5Thread& th, int slot, int gz, int tid) {
    const int base = gz * th.plane;
    if (a.pair8) {
        const int o = base + th.col[0];
        cp_async8(r5_stage_a(stg, slot, 0, tid), a.in0 + o);
        cp_async8(r5_stage_a(stg, slot, 1, tid), a.in1 + o);
        cp_async8(r5_stage_a(stg, slot, 2, tid), a.in2 + o);
    } else {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int o = base + th.col[e];
            cp_async4(r5_stage_a(stg, slot, 0, tid) + e, a.in0 + o);
            cp_async4(r5_stage_a(stg, slot, 1, tid) + e, a.in1 + o);
            cp_async4(r5_stage_a(stg, slot, 2, tid) + e, a.in2 + o);
        }
    }
    cp_async_commit();
}

__device__ __forceinline__ f2 r5_mask(const R5Thread& th, int p, int nz) {
    const float zin = (p >= 0 && p < nz) ? 1.f : 0.f;
    return make_float2(th.cmask.x * zin, th.cmask.y * zin);
}

__device__ __forceinline__ float pick(f2 v, int e) { return e == 0 ? v.x : v.y; }

template <int SEG, bool PREC, int P>
__device__ __forceinline__ void r5_iteration(const Rk5Args& a, R5Rings& r, float* __restrict__ sh,
                                             float* __restrict__ stg, unsigned long long* bars, R5Thread& th, int i,
                                             int t0, int z0, int tid) {
    constexpr int TILE = kTY * kRS;
    float* shb = sh + (P & 1) * (kH * 3 * TILE);
    const int cy0 = th.ty;
    const int cx0 = 2 * th.tx;

    // 1. publish the stage inputs for the y-neighbours
#pragma unroll
    for (int j = 1; j <= kH; ++j) {
        const int slot = (P + kH - j) & 3;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            *reinterpret_cast<f2*>(shb + ((j - 1) * 3 + c) * TILE + cy0 * kRS + cx0) = r.x[j - 1][slot][c];
    }

    // 2. plane t+3 arrives from the staging ring (A: plane t+5 is requested
    //    now; B requests it after the barrier, when no thread still reads
    //    the slot it goes to)
    const int t = i + t0;
    {
        const int slot = (P + kH) & 3;
        if (SEG == 0) {
            r5_issue<SEG>(a, stg, th, (P + kH + 2) & 3, th.gz_issue, tid);
            th.gz_issue = th.gz_issue + 1 == a.nz ? 0 : th.gz_issue + 1;
            cp_async_wait<2>();
#pragma unroll
            for (int c = 0; c < 3; ++c) r.x[0][slot][c] = *reinterpret_cast<const f2*>(r5_stage_a(stg, slot, c, tid));
        } else {
            if (i == 0) mbar_wait(bars + 2, r5_parity(2), a.err, th.bad);   // plane 2: read by stage 4 below
            mbar_wait(bars + slot, r5_parity(i + kH), a.err, th.bad);
            const float4* q = r5_slot_b(reinterpret_cast<const unsigned char*>(stg), slot, th);
            const float4 q0 = q[0], q1 = q[3];
            r.x[0][slot][0] = make_float2(q0.x, q1.x);
            r.x[0][slot][1] = make_float2(q0.y, q1.y);
            r.x[0][slot][2] = make_float2(q0.z, q1.z);
        }
        if (a.bc) {
            const f2 m = r5_mask(th, t + kH, a.nz);
#pragma unroll
            for (int c = 0; c < 3; ++c) r.x[0][slot][c] = mul2(r.x[0][slot][c], m);
        }
    }
    __syncthreads();
    if (SEG == 1 && i + kH + 2 <= a.n_iter + 2) {
        r5_fetch_rows(a, reinterpret_cast<unsigned char*>(stg), bars, th, (P + kH + 2) & 3, th.gz_issue);
        th.gz_issue = th.gz_issue + 1 == a.nz ? 0 : th.gz_issue + 1;
    }

    const int up = cy0 > 0 ? cy0 - 1 : cy0;
    const int dn = cy0 + 1 < kTY ? cy0 + 1 : cy0;
    f2 nb_up[3], nb_dn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        nb_up[c] = *reinterpret_cast<const f2*>(shb + c * TILE + up * kRS + cx0);
        nb_dn[c] = *reinterpret_cast<const f2*>(shb + c * TILE + dn * kRS + cx0);
    }
#pragma unroll
    for (int j = 1; j <= kH; ++j) {
        // warp-uniform: the warp's two rows meet the rows [j, TY-j) where
        // stage j is still needed, and the march has reached its planes
        const bool active = (2 * th.warp_row + 1 >= j) && (2 * th.warp_row < kTY - j) && (i >= 2 * j - 2);
        const int slot = (P + kH - j) & 3;
        const int sm = (slot + 3) & 3, sp = (slot + 1) & 3;
        if (!active) continue;
        f2 cen[3], sum[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const f2 C = r.x[j - 1][slot][c];
            const float L = __shfl_up_sync(0xffffffffu, C.y, 1, kPT);
            const float Rr = __shfl_down_sync(0xffffffffu, C.x, 1, kPT);
            const f2 xs = make_float2(__fadd_rn(L, C.y), __fadd_rn(C.x, Rr));
            sum[c] = add2(add2(add2(xs, add2(nb_up[c], nb_dn[c])), r.x[j - 1][sm][c]), r.x[j - 1][sp][c]);
            cen[c] = C;
        }
        if (j < kH) {
            const float* shn = shb + j * 3 * TILE;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                nb_up[c] = *reinterpret_cast<const f2*>(shn + c * TILE + up * kRS + cx0);
                nb_dn[c] = *reinterpret_cast<const f2*>(shn + c * TILE + dn * kRS + cx0);
            }
        }
        f2 f[3];
        rhs_pair<PREC>(sum, cen, a.J, a.twoD, a.Hx, a.Hy, a.Hz, a.lambda, f);
        const bool emit = j == kH && t >= z0 && t < z0 + a.tz && t < a.nz;
        if (SEG == 0) {
            if (j == 1) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    r.u[slot][c] = f[c];
                    r.x[1][slot][c] = fma2(sp2(a.a21), f[c], r.x[0][slot][c]);
                }
            } else if (j == 2) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    r.v[slot][c] = f[c];
                    r.x[2][slot][c] = fma2(sp2(a.a32), f[c], fma2(sp2(a.a31), r.u[slot][c], r.x[0][slot][c]));
                }
            } else if (emit) {
                f2 x4[3], p5[3], p6[3], py[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const f2 s = r.x[0][slot][c], f1 = r.u[slot][c], g2 = r.v[slot][c], f3 = f[c];
                    x4[c] = fma2(sp2(a.a43), f3, fma2(sp2(a.a42), g2, s));
                    p5[c] = fma2(sp2(a.a51), f1, s);
                    p6[c] = fma2(sp2(a.a63), f3, fma2(sp2(a.a62), g2, fma2(sp2(a.a61), f1, s)));
                    py[c] = fma2(sp2(a.b3), f3, fma2(sp2(a.b1), f1, s));
                }
                // the plane's output records go to shared buffer i & 1; the
                // bulk store that last read it (two planes ago) must be done
                float* ob = stg + 2 * 4 * 3 * kNT + (i & 1) * kOutBufFloats;
                if (th.tx == 0) bulk_wait_read<1>();
                __syncwarp();
                const int ry = th.ty - kH;
                if (ry >= 0 && ry < kOutY) {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int ox = 2 * th.tx + e - kH;
                        if (ox < 0 || ox >= kOutX) continue;
                        float4* dst = reinterpret_cast<float4*>(ob + (ry * kOutX + ox) * kRec);
                        dst[0] = make_float4(pick(x4[0], e), pick(x4[1], e), pick(x4[2], e), pick(p5[0], e));
                        dst[1] = make_float4(pick(p5[1], e), pick(p5[2], e), pick(p6[0], e), pick(p6[1], e));
                        dst[2] = make_float4(pick(p6[2], e), pick(py[0], e), pick(py[1], e), pick(py[2], e));
                    }
                }
                fence_proxy_async();
                __syncwarp();
                if (th.tx == 0 && ry >= 0 && ry < kOutY) {
                    // the row's output sites: columns 26 bx - 1 .. 26 bx + 24
                    // clipped to the lattice (no wrap: the first tile starts
                    // at column 0, the last may stop at the lattice edge)
                    const int gy_u = (int)blockIdx.y * kOutY + ry;
                    const int xw = (int)blockIdx.x * kOutX - kHX + kH;
                    const int off = xw < 0 ? -xw : 0;
                    const int n = min(kOutX - off, a.nx - (xw + off));
                    if (gy_u < a.ny && n > 0) {
                        bulk_s2g(a.car + (size_t)kRec * (unsigned)(t * th.plane + gy_u * a.nx + xw + off),
                                 ob + (ry * kOutX + off) * kRec, (unsigned)(n * kRec * 4));
                        bulk_commit();
                    }
                }
            }
        } else {
            if (j == 1) {
                // stage 4 on plane t+2: its P5, P6, Py are still in the
                // staging slot (the copy for plane t+5 went to another slot)
                const float4* q = r5_slot_b(reinterpret_cast<const unsigned char*>(stg), slot, th);
                const float4 a0 = q[0], a1 = q[1], a2 = q[2], b0 = q[3], b1 = q[4], b2 = q[5];
                f2 p5[3] = {make_float2(a0.w, b0.w), make_float2(a1.x, b1.x), make_float2(a1.y, b1.y)};
                f2 p6[3] = {make_float2(a1.z, b1.z), make_float2(a1.w, b1.w), make_float2(a2.x, b2.x)};
                f2 py[3] = {make_float2(a2.y, b2.y), make_float2(a2.z, b2.z), make_float2(a2.w, b2.w)};
                if (a.bc) {
                    const f2 m = r5_mask(th, t + kH - 1, a.nz);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        p5[c] = mul2(p5[c], m);
                        p6[c] = mul2(p6[c], m);
                        py[c] = mul2(py[c], m);
                    }
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    r.x[1][slot][c] = fma2(sp2(a.a54), f[c], p5[c]);
                    r.u[slot][c] = fma2(sp2(a.a64), f[c], p6[c]);
                    r.v[slot][c] = fma2(sp2(a.b4), f[c], py[c]);
                }
            } else if (j == 2) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    r.x[2][slot][c] = fma2(sp2(a.a65), f[c], r.u[slot][c]);
                    r.v[slot][c] = fma2(sp2(a.b5), f[c], r.v[slot][c]);
                }
            } else if (emit) {
                f2 ox = fma2(sp2(a.b6), f[0], r.v[slot][0]);
                f2 oy = fma2(sp2(a.b6), f[1], r.v[slot][1]);
                f2 oz = fma2(sp2(a.b6), f[2], r.v[slot][2]);
                if (a.renorm) {
                    const f2 n2 = fma2(ox, ox, fma2(oy, oy, mul2(oz, oz)));
                    const f2 inv = make_float2(rsqrtf(n2.x), rsqrtf(n2.y));
                    ox = mul2(ox, inv);
                    oy = mul2(oy, inv);
                    oz = mul2(oz, inv);
                }
                const int base = t * th.plane;
                if (a.pair8 && th.out[0] == th.out[1]) {
                    // both columns of the pair are outputs (or neither): one
                    // 8-byte store per component; the pairs at the window's
                    // edges (tile columns 2-3 and 28-29) store per site
                    if (th.out[0]) {
                        const int site = base + th.col[0];
                        *reinterpret_cast<f2*>(a.out0 + site) = ox;
                        *reinterpret_cast<f2*>(a.out1 + site) = oy;
                        *reinterpret_cast<f2*>(a.out2 + site) = oz;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if (!th.out[e]) continue;
                        const int site = base + th.col[e];
                        a.out0[site] = pick(ox, e);
                        a.out1[site] = pick(oy, e);
                        a.out2[site] = pick(oz, e);
                    }
                }
            }
        }
    }
}

template <int SEG, bool PREC>
__global__ void __launch_bounds__(kNT, 1) k_step_rk5(Rk5Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sh = reinterpret_cast<float*>(smem_raw);
    float* stg = sh + 2 * kH * 3 * kTY * kRS;
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(stg) + 4 * kSlotBytes);
    const int tid = threadIdx.y * kPT + threadIdx.x;
    R5Thread th;
    th.bad = false;
    th.tx = threadIdx.x;
    th.ty = threadIdx.y;
    th.warp_row = __shfl_sync(0xffffffffu, tid >> 5, 0);
    th.plane = a.nx * a.ny;
    {
        const int cy = th.ty;
        const int gyu = (int)blockIdx.y * kOutY - kH + cy;
        const int gy = wrapi(gyu, a.ny);
        th.grow = gy;
        th.gx0 = wrapi((int)blockIdx.x * kOutX - kHX, a.nx);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int cx = 2 * th.tx + e;
            const int gxu = (int)blockIdx.x * kOutX - kHX + cx;
            th.col[e] = gy * a.nx + wrapi(gxu, a.nx);
            th.out[e] = cx >= kH && cx < kH + kOutX && cy >= kH && cy < kTY - kH && gxu >= 0 && gxu < a.nx &&
                        gyu < a.ny;
            const float in = (gxu >= 0 && gxu < a.nx && gyu >= 0 && gyu < a.ny) ? 1.f : 0.f;
            if (e == 0) th.cmask.x = a.bc ? in : 1.f;
            else th.cmask.y = a.bc ? in : 1.f;
        }
    }
    const int z0 = (int)blockIdx.z * a.tz;
    const int t0 = z0 - 2 * kH + 2;

    R5Rings r;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
#pragma unroll
            for (int j = 0; j < 3; ++j) r.x[j][q][c] = make_float2(0.f, 0.f);
            r.u[q][c] = make_float2(0.f, 0.f);
            r.v[q][c] = make_float2(0.f, 0.f);
        }
    // local planes 1 and 2 straight into the first stage's ring
#pragma unroll
    for (int L = 1; L <= 2; ++L) {
        const int base = wrapi(t0 + L, a.nz) * th.plane;
        const int o0 = base + th.col[0], o1 = base + th.col[1];
        if (SEG == 0) {
            r.x[0][L][0] = make_float2(__ldg(a.in0 + o0), __ldg(a.in0 + o1));
            r.x[0][L][1] = make_float2(__ldg(a.in1 + o0), __ldg(a.in1 + o1));
            r.x[0][L][2] = make_float2(__ldg(a.in2 + o0), __ldg(a.in2 + o1));
        } else {
            const float* c0 = a.car + (size_t)kRec * (unsigned)o0;
            const float* c1 = a.car + (size_t)kRec * (unsigned)o1;
            r.x[0][L][0] = make_float2(__ldg(c0 + 0), __ldg(c1 + 0));
            r.x[0][L][1] = make_float2(__ldg(c0 + 1), __ldg(c1 + 1));
            r.x[0][L][2] = make_float2(__ldg(c0 + 2), __ldg(c1 + 2));
        }
        if (a.bc) {
            const f2 m = r5_mask(th, t0 + L, a.nz);
#pragma unroll
            for (int c = 0; c < 3; ++c) r.x[0][L][c] = mul2(r.x[0][L][c], m);
        }
    }
    if (SEG == 1) {
        // the ring's mbarriers: one arrival per tile row and plane
        if (tid == 0)
            for (int q = 0; q < 4; ++q) mbar_init(bars + q, kTY);
        mbar_init_fence();
        __syncthreads();
        // local planes 2 (read by stage 4 at the first iteration), 3 and 4
        r5_fetch_rows(a, reinterpret_cast<unsigned char*>(stg), bars, th, 2, wrapi(t0 + 2, a.nz));
        r5_fetch_rows(a, reinterpret_cast<unsigned char*>(stg), bars, th, 3, wrapi(t0 + 3, a.nz));
        r5_fetch_rows(a, reinterpret_cast<unsigned char*>(stg), bars, th, 0, wrapi(t0 + 4, a.nz));
    } else {
        r5_issue<SEG>(a, stg, th, 3, wrapi(t0 + 3, a.nz), tid);
        r5_issue<SEG>(a, stg, th, 0, wrapi(t0 + 4, a.nz), tid);
    }
    th.gz_issue = wrapi(t0 + 5, a.nz);
    int i = 0;
    for (; i + 4 <= a.n_iter; i += 4) {
        r5_iteration<SEG, PREC, 0>(a, r, sh, stg, bars, th, i + 0, t0, z0, tid);
        r5_iteration<SEG, PREC, 1>(a, r, sh, stg, bars, th, i + 1, t0, z0, tid);
        r5_iteration<SEG, PREC, 2>(a, r, sh, stg, bars, th, i + 2, t0, z0, tid);
        r5_iteration<SEG, PREC, 3>(a, r, sh, stg, bars, th, i + 3, t0, z0, tid);
    }
    if (i < a.n_iter) r5_iteration<SEG, PREC, 0>(a, r, sh, stg, bars, th, i + 0, t0, z0, tid);
    if (i + 1 < a.n_iter) r5_iteration<SEG, PREC, 1>(a, r, sh, stg, bars, th, i + 1, t0, z0, tid);
    if (i + 2 < a.n_iter) r5_iteration<SEG, PREC, 2>(a, r, sh, stg, bars, th, i + 2, t0, z0, tid);
    if (SEG == 0) {
        cp_async_wait<0>();   // no copy may land in shared memory after the tile is done
        if (th.tx == 0) bulk_wait<0>();   // the last record rows are written
    } else {
        // every fetched plane (2 .. n_iter+2) was waited for by the march;
        // after a timeout, wait (bounded) for the copies still in flight
        if (th.bad) {
            th.bad = false;
            for (int p = max(2, a.n_iter - 1); p <= a.n_iter + 2; ++p) mbar_wait(bars + (p & 3), r5_parity(p), nullptr, th.bad);
        }
    }
}

template <int SEG>
constexpr size_t rk5_smem() {
    // y-exchange: 2 buffers x 3 stages x 3 components x tile; then A: the
    // state staging ring (4 slots x 3 components x 8 bytes per thread) and
    // two planes of output records; B: the record ring (4 slots) and its
    // 4 mbarriers
    return sizeof(float) * (size_t)2 * kH * 3 * kTY * kRS +
           (SEG == 0 ? (size_t)4 * 24 * kNT + sizeof(float) * 2 * (size_t)kOutBufFloats
                     : (size_t)4 * kSlotBytes + 4 * sizeof(unsigned long long));
}

template <int SEG, bool PREC>
cudaError_t rk5_launch(const Rk5Args& a, dim3 grid, cudaStream_t st, bool prepare) {
    if (prepare)
        return cudaFuncSetAttribute(k_step_rk5<SEG, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)rk5_smem<SEG>());
    k_step_rk5<SEG, PREC><<<grid, dim3(kPT, kTY), rk5_smem<SEG>(), st>>>(a);
    return cudaGetLastError();
}

// The kernel hard-codes which Butcher coefficients are zero.
bool butcher_rk5_pattern(const Tableau& tb) {
    return tb.stages == 6 && !tb.chain && tb.a[3][0] == 0.0 && tb.a[4][1] == 0.0 && tb.a[4][2] == 0.0 &&
           tb.b[1] == 0.0;
}

}  // namespace

cudaError_t prepare_rk5_kernels() {
    const Rk5Args a{};
    cudaError_t e;
    if ((e = rk5_launch<0, true>(a, dim3(1), 0, true)) != cudaSuccess) return e;
    if ((e = rk5_launch<0, false>(a, dim3(1), 0, true)) != cudaSuccess) return e;
    if ((e = rk5_launch<1, true>(a, dim3(1), 0, true)) != cudaSuccess) return e;
    return rk5_launch<1, false>(a, dim3(1), 0, true);
}

bool rk5_fused_supports(const StepLaunch<float>& L) {
    return butcher_rk5_pattern(*L.tab) && L.hs[0] == nullptr && L.tmp != nullptr && L.st_n[0][0] == nullptr &&
           (reinterpret_cast<uintptr_t>(L.tmp) & 15) == 0;
}

cudaError_t launch_step_rk5(const StepLaunch<float>& L) {
    if (!rk5_fused_supports(L)) return cudaErrorInvalidValue;
    const Tableau& tb = *L.tab;
    Rk5Args a{};
    a.nx = L.g.nx;
    a.ny = L.g.ny;
    a.nz = L.g.nz;
    a.J = L.ph.J;
    a.twoD = L.ph.twoD;
    a.Hx = L.ph.H[0];
    a.Hy = L.ph.H[1];
    a.Hz = L.ph.H[2];
    a.lambda = L.ph.lambda;
    auto c = [&](double v) { return (float)(v * L.dt); };
    a.a21 = c(tb.a[1][0]);
    a.a31 = c(tb.a[2][0]);
    a.a32 = c(tb.a[2][1]);
    a.a42 = c(tb.a[3][1]);
    a.a43 = c(tb.a[3][2]);
    a.a51 = c(tb.a[4][0]);
    a.a54 = c(tb.a[4][3]);
    a.a61 = c(tb.a[5][0]);
    a.a62 = c(tb.a[5][1]);
    a.a63 = c(tb.a[5][2]);
    a.a64 = c(tb.a[5][3]);
    a.a65 = c(tb.a[5][4]);
    a.b1 = c(tb.b[0]);
    a.b3 = c(tb.b[2]);
    a.b4 = c(tb.b[3]);
    a.b5 = c(tb.b[4]);
    a.b6 = c(tb.b[5]);
    a.renorm = L.renorm;
    a.bc = L.bc;
    a.car = L.tmp;   // 12 floats per site in the step scratch
    a.err = L.d_status;
    a.pair8 = pairs_aligned(a.nx, L.in[0], L.in[1], L.in[2]) && pairs_aligned(a.nx, L.out[0], L.out[1], L.out[2]);
    a.in0 = L.in[0];
    a.in1 = L.in[1];
    a.in2 = L.in[2];
    a.out0 = L.out[0];
    a.out1 = L.out[1];
    a.out2 = L.out[2];
    // tile bx outputs columns kOutX bx - 1 .. kOutX bx + kOutX - 2
    const int tiles_x = (L.g.nx + (kHX - kH) + kOutX - 1) / kOutX;
    const int tiles_y = (L.g.ny + kOutY - 1) / kOutY;
    // z chunks: one resident CTA per SM; minimise waves x (chunk planes +
    // pipeline fill of 2 x 3 - 2 iterations)
    const long long tiles = (long long)tiles_x * tiles_y;
    int best_chunks = 1;
    double best_cost = 1e300;
    for (int q = 1; q <= std::max(1, L.g.nz / 4); ++q) {
        const int zc_c = (L.g.nz + q - 1) / q;
        const int used = (L.g.nz + zc_c - 1) / zc_c;
        const double waves = (double)((tiles * used + 151) / 152);
        const double cost = waves * (zc_c + 2 * kH - 2);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best_chunks = q;
        }
    }
    const int zc = (L.g.nz + best_chunks - 1) / best_chunks;
    a.tz = zc;
    a.n_iter = zc + 2 * kH - 2;
    const dim3 grid(tiles_x, tiles_y, (L.g.nz + zc - 1) / zc);
    const bool prec = L.precession != 0;
    cudaError_t e = prec ? rk5_launch<0, true>(a, grid, L.stream, false) : rk5_launch<0, false>(a, grid, L.stream, false);
    if (e != cudaSuccess) return e;
    e = prec ? rk5_launch<1, true>(a, grid, L.stream, false) : rk5_launch<1, false>(a, grid, L.stream, false);
    if (e != cudaSuccess || !L.pulse) return e;
    return launch_pulse_lattice(L);
}

}  // namespace spin
