// Fused FP32 step for chain tableaus (RK4, RK2 midpoint, Heun) with 2x2
// register patches and packed f32x2 arithmetic.
//
// Geometry.  A CTA of 16x16 threads owns a 32x32 tile of lattice columns
// (x, y); each thread owns a 2x2 patch: rows cy = 2ty, 2ty+1, and the column
// pair cx = 2tx, 2tx+1 packed into one float2, so every FP32 operation of the
// right-hand side covers two sites with one f32x2 instruction.  The tile
// carries a halo of S columns (S = stages): after stage j only the columns
// within S-j of the (32-2S)^2 output block are still exact, which is all the
// next stage needs.  The CTA marches along z: at wavefront iteration t it
// streams in spin plane t+S and evaluates stage j on plane t+S-j, so every
// stage state lives on chip for exactly the planes its z-neighbours need
// (per-thread register rings indexed by plane & 3).
//
// Neighbour exchange per stage: x-neighbours by warp shuffles inside each
// 16-lane row segment, y-neighbours through shared memory (one double-
// buffered plane per stage, one barrier per iteration), z-neighbours from
// the rings.  One HBM read and one write of the state per step; the pulse
// rotation (Eq. s_rotation) runs in the epilogue of its step.
#include <cuda_runtime.h>

#include <algorithm>

#include "patch_common.cuh"
#include "spin_device.cuh"
#include "spin_internal.h"

namespace spin {

namespace {

// Rows per thread (PY) and thread rows (TY) per stage count and tile variant
// V: RK4 keeps one row per thread (register rings of 4 stage planes do not fit
// twice), RK2/Heun two.  Variant 0 is the single-lattice tile; the batched
// replicas choose among the variants per replica size (the tile's output
// height is PY*TY - 2S rows, and a replica of side L needs ceil(L/out) tiles
// along y).
template <int S, int V = 0>
struct PatchShape;
#ifndef SPIN_PATCH_TY4
#define SPIN_PATCH_TY4 24
#endif
template <>
struct PatchShape<4, 0> {
    static constexpr int PY = 1, TY = SPIN_PATCH_TY4;
};
template <>
struct PatchShape<4, 1> {
    static constexpr int PY = 1, TY = 20;
};
template <>
struct PatchShape<4, 2> {
    static constexpr int PY = 1, TY = 16;
};
template <>
struct PatchShape<2, 0> {
    static constexpr int PY = 2, TY = 16;
};
template <>
struct PatchShape<2, 1> {
    static constexpr int PY = 2, TY = 12;
};
template <>
struct PatchShape<2, 2> {
    static constexpr int PY = 2, TY = 8;
};
constexpr int kTileVariants = 3;

struct PatchArgs {
    const float* __restrict__ in0;
    const float* __restrict__ in1;
    const float* __restrict__ in2;
    float* __restrict__ out0;
    float* __restrict__ out1;
    float* __restrict__ out2;
    const float* __restrict__ hs0;
    const float* __restrict__ hs1;
    const float* __restrict__ hs2;
    int nx, ny, nz, tz, n_iter;
    float J, twoD, Hx, Hy, Hz, lambda;
    float cdt[4];
    float bdt[4];
    int renorm;
    uint64_t seed, replica;
    float sigma;
    const long long* interval;
    int bc;            // 1: free boundaries (outside columns and planes read as zero spins)
    int pair8;         // 1: each thread's column pair is one aligned 8-byte word of every input plane
    int pair8out;      // 1: the same for the output planes
    // stage store (STORE variant, for the adjoint's recomputation): at the
    // output sites, the stage inputs X_j (j = 2..S, stx[j-2]), the stage
    // neighbour sums sum_nn X_j (j = 1..S, stn[j-1]) and the unnormalised RK
    // result y (sty), component arrays in the lattice's layout
    float* stx[3][3];
    float* stn[4][3];
    float* sty[3];
    float dt;
    int* err;          // device status word for bounded waits (nullable; no wait in this kernel sets it)
};

template <int S, bool HSITE>
struct PRings {
    static constexpr int PY = PatchShape<S>::PY;
    f2 s[4][PY][3];
    f2 x[S - 1][4][PY][3];
    f2 y[4][PY][3];
    f2 h[HSITE ? 4 : 1][PY][3];
};

template <int PY>
struct PThread {
    int tx, ty, warp_row;
    int col[PY][2];    // [row][pair element] global column index gy*nx+gx
    bool out[PY][2];
    int plane;         // nx*ny
    int gz_issue;      // wrapped z of the next plane to prefetch (t+S+2)
    int gz_field;      // wrapped z of the next site-field plane (t+S-1)
    f2 cmask[PY];      // 1 for lattice columns, 0 for columns outside a free-boundary lattice
};

// Per-thread staging ring for spin planes fetched two iterations ahead with
// cp.async (the thread only ever reads back its own columns): 4 slots x 3
// components x PY rows, one column pair (two adjacent floats) per thread,
// thread-minor, so the pair is one conflict-free 8-byte access.
template <int S, int V>
__device__ __forceinline__ float* stage_pair(float* stg, int slot, int c, int rr, int tid) {
    constexpr int PY = PatchShape<S, V>::PY, NT = kPT * PatchShape<S, V>::TY;
    return stg + 2 * ((((slot * 3 + c) * PY + rr) * NT) + tid);
}

template <int S, int V>
__device__ __forceinline__ void issue_plane(const PatchArgs& a, float* stg, const PThread<PatchShape<S>::PY>& th,
                                            int slot, int gz, int tid) {
    constexpr int PY = PatchShape<S>::PY;
    const int base = gz * th.plane;   // site offsets fit in 32 bits (N < 2^31)
    if (a.pair8) {
#pragma unroll
        for (int rr = 0; rr < PY; ++rr) {
            const int o = base + th.col[rr][0];
            cp_async8(stage_pair<S, V>(stg, slot, 0, rr, tid), a.in0 + o);
            cp_async8(stage_pair<S, V>(stg, slot, 1, rr, tid), a.in1 + o);
            cp_async8(stage_pair<S, V>(stg, slot, 2, rr, tid), a.in2 + o);
        }
    } else {
#pragma unroll
        for (int rr = 0; rr < PY; ++rr)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int o = base + th.col[rr][e];
                cp_async4(stage_pair<S, V>(stg, slot, 0, rr, tid) + e, a.in0 + o);
                cp_async4(stage_pair<S, V>(stg, slot, 1, rr, tid) + e, a.in1 + o);
                cp_async4(stage_pair<S, V>(stg, slot, 2, rr, tid) + e, a.in2 + o);
            }
    }
    cp_async_commit();
}

template <int S, bool PREC, bool HSITE, bool PULSE, bool STORE, int P, int V>
__device__ __forceinline__ void patch_iteration(const PatchArgs& a, PRings<S, HSITE>& r, float* __restrict__ sh,
                                                float* __restrict__ stg, PThread<PatchShape<S>::PY>& th, int i,
                                                int t0, int z0, long long k, int tid) {
    constexpr int PY = PatchShape<S, V>::PY, ROWS = PatchShape<S, V>::PY * PatchShape<S, V>::TY;
    constexpr int TILE = ROWS * kRS;
    float* shb = sh + (P & 1) * (S * 3 * TILE);
    const int cy0 = PY * th.ty;
    const int cx0 = 2 * th.tx;

    // 1. publish the stage inputs (both rows) for the y-neighbours
#pragma unroll
    for (int j = 1; j <= S; ++j) {
        const int slot = (P + S - j) & 3;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int rr = 0; rr < PY; ++rr) {
                const f2 v = (j == 1) ? r.s[slot][rr][c] : r.x[j - 2][slot][rr][c];
                *reinterpret_cast<f2*>(shb + ((j - 1) * 3 + c) * TILE + (cy0 + rr) * kRS + cx0) = v;
            }
    }

    // 2. spin plane t+S arrives from the staging ring (fetched two iterations
    //    ago); plane t+S+2 is requested now
    const int t = i + t0;
    {
        issue_plane<S, V>(a, stg, th, (P + S + 2) & 3, th.gz_issue, tid);
        th.gz_issue = th.gz_issue + 1 == a.nz ? 0 : th.gz_issue + 1;
        cp_async_wait<2>();
        const int slot = (P + S) & 3;
#pragma unroll
        for (int rr = 0; rr < PY; ++rr)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                r.s[slot][rr][c] = *reinterpret_cast<const f2*>(stage_pair<S, V>(stg, slot, c, rr, tid));
        if (a.bc) {
            // free boundaries: no spin outside the lattice (a zero spin stays
            // zero through every stage, so it never feeds the stencil)
            const float zin = (t + S >= 0 && t + S < a.nz) ? 1.f : 0.f;
#pragma unroll
            for (int rr = 0; rr < PY; ++rr) {
                const f2 m = make_float2(th.cmask[rr].x * zin, th.cmask[rr].y * zin);
#pragma unroll
                for (int c = 0; c < 3; ++c) r.s[slot][rr][c] = mul2(r.s[slot][rr][c], m);
            }
        }
        if (HSITE) {
            const int bh = th.gz_field * th.plane;
            th.gz_field = th.gz_field + 1 == a.nz ? 0 : th.gz_field + 1;
            const int sl = (P + S - 1) & 3;
#pragma unroll
            for (int rr = 0; rr < PY; ++rr) {
                const int o0 = bh + th.col[rr][0], o1 = bh + th.col[rr][1];
                r.h[sl][rr][0] = make_float2(__ldg(a.hs0 + o0), __ldg(a.hs0 + o1));
                r.h[sl][rr][1] = make_float2(__ldg(a.hs1 + o0), __ldg(a.hs1 + o1));
                r.h[sl][rr][2] = make_float2(__ldg(a.hs2 + o0), __ldg(a.hs2 + o1));
            }
        }
    }
    __syncthreads();

    const int up = cy0 > 0 ? cy0 - 1 : cy0;                     // row above the first row (clamped at the tile edge)
    const int dn = cy0 + PY < ROWS ? cy0 + PY : cy0 + PY - 1;   // row below the last row

    // 3. stage j on plane t+S-j; the rows above and below for stage j+1 are
    //    requested from shared memory before stage j's arithmetic
    f2 nb_up[3], nb_dn[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        nb_up[c] = *reinterpret_cast<const f2*>(shb + c * TILE + up * kRS + cx0);
        nb_dn[c] = *reinterpret_cast<const f2*>(shb + c * TILE + dn * kRS + cx0);
    }
#pragma unroll
    for (int j = 1; j <= S; ++j) {
        // the 2*PY rows of warp w take part in stage j only if they meet the
        // rows [j, ROWS-j) where stage j is still needed, and only once the
        // march has reached the planes stage j is needed on: stage j serves
        // planes z0-(S-j) .. z0+tz+(S-j)-1, which it reaches at iteration
        // i = 2j-2 (earlier iterations would compute planes no later stage
        // reads; the test is warp-uniform)
        const bool active = (2 * PY * th.warp_row + 2 * PY - 1 >= j) && (2 * PY * th.warp_row < ROWS - j) &&
                            (i >= 2 * j - 2);
        const int slot = (P + S - j) & 3;
        const int sm = (slot + 3) & 3, sp = (slot + 1) & 3;
        if (active) {
            f2 cen[PY][3], sum[PY][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const f2 row_up = nb_up[c];
                const f2 row_dn = nb_dn[c];
#pragma unroll
                for (int rr = 0; rr < PY; ++rr) {
                    const f2 C = (j == 1) ? r.s[slot][rr][c] : r.x[j - 2][slot][rr][c];
                    const f2 ZM = (j == 1) ? r.s[sm][rr][c] : r.x[j - 2][sm][rr][c];
                    const f2 ZP = (j == 1) ? r.s[sp][rr][c] : r.x[j - 2][sp][rr][c];
                    // x-neighbours: left of the pair's first column and right of its second
                    const float L = __shfl_up_sync(0xffffffffu, C.y, 1, kPT);
                    const float Rr = __shfl_down_sync(0xffffffffu, C.x, 1, kPT);
                    // (x-1) + (x+1) for both columns of the pair, as two scalar adds
                    const f2 xs = make_float2(__fadd_rn(L, C.y), __fadd_rn(C.x, Rr));
                    const int ro = PY == 2 ? (rr ^ 1) : rr;
                    const f2 other = (j == 1) ? r.s[slot][ro][c] : r.x[j - 2][slot][ro][c];
                    const f2 ym = rr == 0 ? row_up : other;
                    const f2 yp = rr == PY - 1 ? row_dn : other;
                    // ((x-1 + x+1) + (y-1 + y+1)) + z-1, and z+1 last: it is the
                    // value the previous stage produced in this iteration
                    sum[rr][c] = add2(add2(add2(xs, add2(ym, yp)), ZM), ZP);
                    cen[rr][c] = C;
                }
            }
            if (j < S) {
                const float* shn = shb + j * 3 * TILE;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    nb_up[c] = *reinterpret_cast<const f2*>(shn + c * TILE + up * kRS + cx0);
                    nb_dn[c] = *reinterpret_cast<const f2*>(shn + c * TILE + dn * kRS + cx0);
                }
            }
#pragma unroll
            for (int rr = 0; rr < PY; ++rr) {
                f2 hx = fma2(sp2(a.J), sum[rr][0], sp2(a.Hx));
                f2 hy = fma2(sp2(a.J), sum[rr][1], sp2(a.Hy));
                f2 hz = fma2(sp2(a.J), sum[rr][2], sp2(a.Hz));
                if (HSITE) {
                    hx = add2(hx, r.h[slot][rr][0]);
                    hy = add2(hy, r.h[slot][rr][1]);
                    hz = add2(hz, r.h[slot][rr][2]);
                }
                const f2 sx = cen[rr][0], sy = cen[rr][1], sz = cen[rr][2];
                hz = fma2(sp2(a.twoD), sz, hz);
                // a = s x H ; b = s x a ; f = a - lambda b  (slow: f = -lambda b)
                const f2 nx_ = make_float2(-sx.x, -sx.y), ny_ = make_float2(-sy.x, -sy.y), nz_ = make_float2(-sz.x, -sz.y);
                const f2 ax = fma2(nz_, hy, mul2(sy, hz));
                const f2 ay = fma2(nx_, hz, mul2(sz, hx));
                const f2 az = fma2(ny_, hx, mul2(sx, hy));
                const f2 bx = fma2(nz_, ay, mul2(sy, az));
                const f2 by = fma2(nx_, az, mul2(sz, ax));
                const f2 bz = fma2(ny_, ax, mul2(sx, ay));
                f2 f[3];
                if (PREC) {
                    f[0] = fma2(sp2(-a.lambda), bx, ax);
                    f[1] = fma2(sp2(-a.lambda), by, ay);
                    f[2] = fma2(sp2(-a.lambda), bz, az);
                } else {
                    f[0] = mul2(sp2(-a.lambda), bx);
                    f[1] = mul2(sp2(-a.lambda), by);
                    f[2] = mul2(sp2(-a.lambda), bz);
                }
                if (STORE) {
                    // stage input and neighbour sum of plane t+S-j at the output sites
                    const int pz = t + S - j;
                    if (pz >= z0 && pz < z0 + a.tz && pz < a.nz) {
                        const int base = pz * th.plane;
                        if (a.pair8out) {
                            // both columns of the pair are outputs or neither: 8-byte stores
                            if (th.out[rr][0]) {
                                const int site = base + th.col[rr][0];
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    *reinterpret_cast<f2*>(a.stn[j - 1][c] + site) = sum[rr][c];
                                    if (j >= 2) *reinterpret_cast<f2*>(a.stx[j >= 2 ? j - 2 : 0][c] + site) = cen[rr][c];
                                }
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                if (!th.out[rr][e]) continue;
                                const int site = base + th.col[rr][e];
#pragma unroll
                                for (int c = 0; c < 3; ++c) {
                                    a.stn[j - 1][c][site] = e == 0 ? sum[rr][c].x : sum[rr][c].y;
                                    if (j >= 2) a.stx[j >= 2 ? j - 2 : 0][c][site] = e == 0 ? cen[rr][c].x : cen[rr][c].y;
                                }
                            }
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (j == 1)
                        r.y[slot][rr][c] = fma2(sp2(a.bdt[0]), f[c], r.s[slot][rr][c]);
                    else
                        r.y[slot][rr][c] = fma2(sp2(a.bdt[j - 1]), f[c], r.y[slot][rr][c]);
                    if (j < S) r.x[j - 1][slot][rr][c] = fma2(sp2(a.cdt[j - 1]), f[c], r.s[slot][rr][c]);
                }
            }
        }
        if (j == S && active && t >= z0 && t < z0 + a.tz && t < a.nz) {
            // finished plane t: renormalise, pulse, store
            const int base = t * th.plane;
#pragma unroll
            for (int rr = 0; rr < PY; ++rr) {
                f2 ox = r.y[slot][rr][0], oy = r.y[slot][rr][1], oz = r.y[slot][rr][2];
                if (STORE) {
                    // the unnormalised RK result, for the adjoint's renormalisation transpose
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if (!th.out[rr][e]) continue;
                        const int site = base + th.col[rr][e];
                        a.sty[0][site] = e == 0 ? ox.x : ox.y;
                        a.sty[1][site] = e == 0 ? oy.x : oy.y;
                        a.sty[2][site] = e == 0 ? oz.x : oz.y;
                    }
                }
                if (a.renorm) {
                    const f2 n2 = fma2(ox, ox, fma2(oy, oy, mul2(oz, oz)));
                    const f2 inv = make_float2(rsqrtf(n2.x), rsqrtf(n2.y));
                    ox = mul2(ox, inv);
                    oy = mul2(oy, inv);
                    oz = mul2(oz, inv);
                }
                if (!PULSE && a.pair8out) {
                    // both columns of the pair are outputs or neither (even row
                    // length, even tile offsets): one 8-byte store per component
                    if (th.out[rr][0]) {
                        const int site = base + th.col[rr][0];
                        *reinterpret_cast<f2*>(a.out0 + site) = ox;
                        *reinterpret_cast<f2*>(a.out1 + site) = oy;
                        *reinterpret_cast<f2*>(a.out2 + site) = oz;
                    }
                    continue;
                }
                float vx[2] = {ox.x, ox.y}, vy[2] = {oy.x, oy.y}, vz[2] = {oz.x, oz.y};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (!th.out[rr][e]) continue;
                    const int site = base + th.col[rr][e];
                    if (PULSE) pulse_site<float>(vx[e], vy[e], vz[e], a.seed, (uint64_t)site, (uint64_t)k, a.replica, a.sigma);
                    a.out0[site] = vx[e];
                    a.out1[site] = vy[e];
                    a.out2[site] = vz[e];
                }
            }
        }
    }
}

// One CTA's tile: columns (bx, by) of the x-y tiling, z chunk bz.
template <int S, bool PREC, bool HSITE, bool PULSE, bool STORE, int V>
__device__ __forceinline__ void patch_tile(const PatchArgs& a, int bx, int by, int bz, float* __restrict__ sh) {
    constexpr int PY = PatchShape<S, V>::PY, ROWS = PatchShape<S, V>::PY * PatchShape<S, V>::TY;
    float* stg = sh + 2 * S * 3 * ROWS * kRS;
    const int tid = threadIdx.y * kPT + threadIdx.x;
    PThread<PY> th;
    th.tx = threadIdx.x;
    th.ty = threadIdx.y;
    // two thread rows per warp; broadcast from lane 0 so that the compiler
    // knows the index (and every stage-activity test built on it) is
    // warp-uniform and branches without divergence handling
    th.warp_row = __shfl_sync(0xffffffffu, (int)((threadIdx.y * kPT + threadIdx.x) >> 5), 0);
    constexpr int OUTX = kPC - 2 * S, OUTY = ROWS - 2 * S;
    th.plane = a.nx * a.ny;
#pragma unroll
    for (int rr = 0; rr < PY; ++rr) {
        const int cy = PY * th.ty + rr;
        const int gyu = by * OUTY - S + cy;
        const int gy = wrapi(gyu, a.ny);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int cx = 2 * th.tx + e;
            const int gxu = bx * OUTX - S + cx;
            th.col[rr][e] = gy * a.nx + wrapi(gxu, a.nx);
            th.out[rr][e] = cx >= S && cx < kPC - S && cy >= S && cy < ROWS - S && gxu < a.nx && gyu < a.ny;
            const float in = (gxu >= 0 && gxu < a.nx && gyu >= 0 && gyu < a.ny) ? 1.f : 0.f;
            if (e == 0) th.cmask[rr].x = a.bc ? in : 1.f;
            else th.cmask[rr].y = a.bc ? in : 1.f;
        }
    }
    const int z0 = bz * a.tz;
    const int t0 = z0 - 2 * S + 2;
    const long long k = PULSE ? *a.interval : 0;

    PRings<S, HSITE> r;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int rr = 0; rr < PY; ++rr)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                r.s[q][rr][c] = make_float2(0.f, 0.f);
                r.y[q][rr][c] = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < S - 1; ++j) r.x[j][q][rr][c] = make_float2(0.f, 0.f);
                if (HSITE) r.h[q][rr][c] = make_float2(0.f, 0.f);
            }
#pragma unroll
    for (int L = S - 2; L <= S - 1; ++L) {
        const int base = wrapi(t0 + L, a.nz) * th.plane;
#pragma unroll
        for (int rr = 0; rr < PY; ++rr) {
            const int o0 = base + th.col[rr][0], o1 = base + th.col[rr][1];
            r.s[L & 3][rr][0] = make_float2(__ldg(a.in0 + o0), __ldg(a.in0 + o1));
            r.s[L & 3][rr][1] = make_float2(__ldg(a.in1 + o0), __ldg(a.in1 + o1));
            r.s[L & 3][rr][2] = make_float2(__ldg(a.in2 + o0), __ldg(a.in2 + o1));
            if (a.bc) {
                const float zin = (t0 + L >= 0 && t0 + L < a.nz) ? 1.f : 0.f;
                const f2 m = make_float2(th.cmask[rr].x * zin, th.cmask[rr].y * zin);
#pragma unroll
                for (int c = 0; c < 3; ++c) r.s[L & 3][rr][c] = mul2(r.s[L & 3][rr][c], m);
            }
        }
    }
    // planes S and S+1 (local) go to the staging ring before the march
    issue_plane<S, V>(a, stg, th, S & 3, wrapi(t0 + S, a.nz), tid);
    issue_plane<S, V>(a, stg, th, (S + 1) & 3, wrapi(t0 + S + 1, a.nz), tid);
    th.gz_issue = wrapi(t0 + S + 2, a.nz);
    th.gz_field = wrapi(t0 + S - 1, a.nz);
    int i = 0;
    for (; i + 4 <= a.n_iter; i += 4) {
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 0, V>(a, r, sh, stg, th, i + 0, t0, z0, k, tid);
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 1, V>(a, r, sh, stg, th, i + 1, t0, z0, k, tid);
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 2, V>(a, r, sh, stg, th, i + 2, t0, z0, k, tid);
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 3, V>(a, r, sh, stg, th, i + 3, t0, z0, k, tid);
    }
    if (i < a.n_iter) patch_iteration<S, PREC, HSITE, PULSE, STORE, 0, V>(a, r, sh, stg, th, i + 0, t0, z0, k, tid);
    if (i + 1 < a.n_iter) patch_iteration<S, PREC, HSITE, PULSE, STORE, 1, V>(a, r, sh, stg, th, i + 1, t0, z0, k, tid);
    if (i + 2 < a.n_iter) patch_iteration<S, PREC, HSITE, PULSE, STORE, 2, V>(a, r, sh, stg, th, i + 2, t0, z0, k, tid);
    cp_async_wait<0>();   // no copy may land in shared memory after the tile is done
}

template <int S, bool PREC, bool HSITE, bool PULSE>
__global__ void __launch_bounds__(kPT* PatchShape<S>::TY, 1) k_step_patch(PatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    patch_tile<S, PREC, HSITE, PULSE, false, 0>(a, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                                             reinterpret_cast<float*>(smem_raw));
}

// The same step that also writes every stage's input and increment at the
// output sites (the adjoint reads them instead of recomputing the stages).
template <int S, bool PREC, bool HSITE>
__global__ void __launch_bounds__(kPT* PatchShape<S>::TY, 1) k_step_patch_store(PatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    patch_tile<S, PREC, HSITE, false, true, 0>(a, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                                            reinterpret_cast<float*>(smem_raw));
}

// Batched replicas: one CTA per work item (replica, x tile, y tile, z chunk)
// of a table sorted by cost; each replica is a cubic periodic lattice of side
// L at its own offset in the concatenated arrays, with its own pulse angle
// scale (temperature) and its index as the noise counter's replica word.
template <int S, bool PREC, bool PULSE, int V>
__global__ void __launch_bounds__(kPT* PatchShape<S, V>::TY, 1)
    k_step_patch_batch(PatchArgs base, const BatchItem* __restrict__ items, const BatchRep* __restrict__ reps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchItem it = items[blockIdx.x];
    const BatchRep rp = reps[it.rep];
    PatchArgs a = base;
    a.in0 += rp.off;
    a.in1 += rp.off;
    a.in2 += rp.off;
    a.out0 += rp.off;
    a.out1 += rp.off;
    a.out2 += rp.off;
    a.nx = a.ny = a.nz = rp.L;
    a.pair8 = pairs_aligned(rp.L, a.in0, a.in1, a.in2) ? 1 : 0;
    a.pair8out = pairs_aligned(rp.L, a.out0, a.out1, a.out2) ? 1 : 0;
    a.tz = rp.tz;
    a.n_iter = rp.tz + 2 * S - 2;
    a.sigma = rp.sigma;
    a.replica = (uint64_t)it.rep;
    patch_tile<S, PREC, false, PULSE, false, V>(a, it.bx, it.by, it.bz, reinterpret_cast<float*>(smem_raw));
}

template <int S, bool PREC, bool HSITE, bool PULSE, int V = 0>
size_t patch_smem() {
    constexpr int ROWS = PatchShape<S, V>::PY * PatchShape<S, V>::TY, NT = kPT * PatchShape<S, V>::TY;
    return sizeof(float) * (2 * S * 3 * ROWS * kRS + 4 * 3 * PatchShape<S, V>::PY * 2 * NT);
}

template <int S, bool PREC, bool HSITE, bool PULSE>
cudaError_t patch_launch(const PatchArgs& a, dim3 grid, cudaStream_t st, bool prepare) {
    const size_t smem = patch_smem<S, PREC, HSITE, PULSE>();
    if (prepare)
        return cudaFuncSetAttribute(k_step_patch<S, PREC, HSITE, PULSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    k_step_patch<S, PREC, HSITE, PULSE><<<grid, dim3(kPT, PatchShape<S>::TY), smem, st>>>(a);
    return cudaGetLastError();
}

template <int S, bool PREC, bool HSITE>
cudaError_t patch_store_launch(const PatchArgs& a, dim3 grid, cudaStream_t st, bool prepare) {
    const size_t smem = patch_smem<S, PREC, HSITE, false>();
    if (prepare)
        return cudaFuncSetAttribute(k_step_patch_store<S, PREC, HSITE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    k_step_patch_store<S, PREC, HSITE><<<grid, dim3(kPT, PatchShape<S>::TY), smem, st>>>(a);
    return cudaGetLastError();
}

template <int S>
cudaError_t patch_store_dispatch(const PatchArgs& a, dim3 grid, cudaStream_t st, bool prec, bool hs, bool prepare) {
    if (prepare) {
        cudaError_t e;
        if ((e = patch_store_launch<S, true, false>(a, grid, st, true)) != cudaSuccess) return e;
        if ((e = patch_store_launch<S, true, true>(a, grid, st, true)) != cudaSuccess) return e;
        if ((e = patch_store_launch<S, false, false>(a, grid, st, true)) != cudaSuccess) return e;
        return patch_store_launch<S, false, true>(a, grid, st, true);
    }
    if (prec) return hs ? patch_store_launch<S, true, true>(a, grid, st, false)
                        : patch_store_launch<S, true, false>(a, grid, st, false);
    return hs ? patch_store_launch<S, false, true>(a, grid, st, false) : patch_store_launch<S, false, false>(a, grid, st, false);
}

template <int S>
cudaError_t patch_dispatch(const PatchArgs& a, dim3 grid, cudaStream_t st, bool prec, bool hs, bool pulse,
                           bool prepare) {
#define SPIN_PATCH_CASE(P_, H_, U_)                                                   \
    if (prepare) {                                                                    \
        cudaError_t e = patch_launch<S, P_, H_, U_>(a, grid, st, true);               \
        if (e != cudaSuccess) return e;                                               \
    } else if (prec == P_ && hs == H_ && pulse == U_) {                               \
        return patch_launch<S, P_, H_, U_>(a, grid, st, false);                       \
    }
    SPIN_PATCH_CASE(true, false, false)
    SPIN_PATCH_CASE(true, false, true)
    SPIN_PATCH_CASE(true, true, false)
    SPIN_PATCH_CASE(true, true, true)
    SPIN_PATCH_CASE(false, false, false)
    SPIN_PATCH_CASE(false, false, true)
    SPIN_PATCH_CASE(false, true, false)
    SPIN_PATCH_CASE(false, true, true)
#undef SPIN_PATCH_CASE
    return prepare ? cudaSuccess : cudaErrorInvalidValue;
}

template <int S, bool PREC, bool PULSE, int V>
cudaError_t batch_launch(const PatchArgs& a, const BatchItem* items, int nitems, const BatchRep* reps, cudaStream_t st,
                         bool prepare) {
    const size_t smem = patch_smem<S, PREC, false, PULSE, V>();
    if (prepare)
        return cudaFuncSetAttribute(k_step_patch_batch<S, PREC, PULSE, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    if (nitems <= 0) return cudaSuccess;
    k_step_patch_batch<S, PREC, PULSE, V><<<nitems, dim3(kPT, PatchShape<S, V>::TY), smem, st>>>(a, items, reps);
    return cudaGetLastError();
}

template <int S, int V>
cudaError_t batch_dispatch_v(const PatchArgs& a, const BatchItem* items, int nitems, const BatchRep* reps,
                             cudaStream_t st, bool prec, bool pulse, bool prepare) {
    if (prepare) {
        cudaError_t e;
        if ((e = batch_launch<S, true, false, V>(a, items, nitems, reps, st, true)) != cudaSuccess) return e;
        if ((e = batch_launch<S, true, true, V>(a, items, nitems, reps, st, true)) != cudaSuccess) return e;
        if ((e = batch_launch<S, false, false, V>(a, items, nitems, reps, st, true)) != cudaSuccess) return e;
        return batch_launch<S, false, true, V>(a, items, nitems, reps, st, true);
    }
    if (prec) return pulse ? batch_launch<S, true, true, V>(a, items, nitems, reps, st, false)
                           : batch_launch<S, true, false, V>(a, items, nitems, reps, st, false);
    return pulse ? batch_launch<S, false, true, V>(a, items, nitems, reps, st, false)
                 : batch_launch<S, false, false, V>(a, items, nitems, reps, st, false);
}

template <int S>
cudaError_t batch_dispatch(const PatchArgs& a, const BatchItem* items, int nitems, const BatchRep* reps,
                           cudaStream_t st, bool prec, bool pulse, bool prepare, int variant) {
    if (prepare) {
        cudaError_t e;
        if ((e = batch_dispatch_v<S, 0>(a, items, nitems, reps, st, prec, pulse, true)) != cudaSuccess) return e;
        if ((e = batch_dispatch_v<S, 1>(a, items, nitems, reps, st, prec, pulse, true)) != cudaSuccess) return e;
        return batch_dispatch_v<S, 2>(a, items, nitems, reps, st, prec, pulse, true);
    }
    switch (variant) {
        case 0: return batch_dispatch_v<S, 0>(a, items, nitems, reps, st, prec, pulse, false);
        case 1: return batch_dispatch_v<S, 1>(a, items, nitems, reps, st, prec, pulse, false);
        case 2: return batch_dispatch_v<S, 2>(a, items, nitems, reps, st, prec, pulse, false);
        default: return cudaErrorInvalidValue;
    }
}

PatchArgs patch_args_common(const StepLaunch<float>& L) {
    const Tableau& tb = *L.tab;
    const int S = tb.stages;
    PatchArgs a{};
    a.in0 = L.in[0];
    a.in1 = L.in[1];
    a.in2 = L.in[2];
    a.out0 = L.out[0];
    a.out1 = L.out[1];
    a.out2 = L.out[2];
    a.hs0 = L.hs[0];
    a.hs1 = L.hs[1];
    a.hs2 = L.hs[2];
    a.nx = L.g.nx;
    a.ny = L.g.ny;
    a.nz = L.g.nz;
    a.J = L.ph.J;
    a.twoD = L.ph.twoD;
    a.Hx = L.ph.H[0];
    a.Hy = L.ph.H[1];
    a.Hz = L.ph.H[2];
    a.lambda = L.ph.lambda;
    for (int j = 0; j < 4; ++j) {
        a.cdt[j] = (j + 1 < S) ? (float)(tb.a[j + 1][j] * L.dt) : 0.f;
        a.bdt[j] = (j < S) ? (float)(tb.b[j] * L.dt) : 0.f;
    }
    a.renorm = L.renorm;
    a.seed = L.seed;
    a.replica = L.replica;
    a.pair8 = pairs_aligned(a.nx, a.in0, a.in1, a.in2) ? 1 : 0;
    a.pair8out = pairs_aligned(a.nx, a.out0, a.out1, a.out2) ? 1 : 0;
    a.sigma = L.sigma;
    a.interval = L.d_interval;
    a.bc = L.bc;
    a.err = L.d_status;
    return a;
}

// The noise pulse on its own, over every site of the lattice (all threads
// busy): on pulse steps of a single lattice the step kernel runs without its
// epilogue rotation and this kernel rotates the finished state in place.  The
// arithmetic per site is the fused epilogue's, so the results are identical.
__global__ void __launch_bounds__(256) k_pulse_f32(float* __restrict__ sx, float* __restrict__ sy, float* __restrict__ sz,
                                                   long long N, uint64_t seed, const long long* __restrict__ interval,
                                                   uint64_t replica, float sigma) {
    const uint64_t k = (uint64_t)*interval;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float x = sx[i], y = sy[i], z = sz[i];
        pulse_site<float>(x, y, z, seed, (uint64_t)i, k, replica, sigma);
        sx[i] = x;
        sy[i] = y;
        sz[i] = z;
    }
}

// Batched pulse: block b rotates the sites of rows [row0, row0+nrows) of
// replica rep (the observables' block table), with that replica's angle scale
// and noise stream; same per-site arithmetic as the single-lattice kernel.
__global__ void __launch_bounds__(256) k_pulse_batch(float* __restrict__ sx, float* __restrict__ sy,
                                                     float* __restrict__ sz, const BatchRep* __restrict__ reps,
                                                     const ObsBlock* __restrict__ blocks, uint64_t seed,
                                                     const long long* __restrict__ interval) {
    const ObsBlock ob = blocks[blockIdx.x];
    const BatchRep rp = reps[ob.rep];
    const uint64_t k = (uint64_t)*interval;
    const long long first = (long long)ob.row0 * rp.L;
    const long long count = (long long)ob.nrows * rp.L;
    for (long long q = threadIdx.x; q < count; q += blockDim.x) {
        const long long i = first + q;          // site index within the replica
        const long long g = rp.off + i;
        float x = sx[g], y = sy[g], z = sz[g];
        pulse_site<float>(x, y, z, seed, (uint64_t)i, k, (uint64_t)ob.rep, rp.sigma);
        sx[g] = x;
        sy[g] = y;
        sz[g] = z;
    }
}

}  // namespace

cudaError_t launch_pulse_batch(float* s[3], const BatchRep* reps, const ObsBlock* blocks, int nblocks, uint64_t seed,
                               const long long* d_interval, cudaStream_t st) {
    k_pulse_batch<<<nblocks, 256, 0, st>>>(s[0], s[1], s[2], reps, blocks, seed, d_interval);
    return cudaGetLastError();
}

int patch_out_x(int stages) { return kPC - 2 * stages; }
int patch_rows(int stages, int variant) {
    if (stages == 4)
        return variant == 1 ? PatchShape<4, 1>::TY : (variant == 2 ? PatchShape<4, 2>::TY : PatchShape<4, 0>::TY);
    return PatchShape<2, 0>::PY *
           (variant == 1 ? PatchShape<2, 1>::TY : (variant == 2 ? PatchShape<2, 2>::TY : PatchShape<2, 0>::TY));
}
int patch_out_y(int stages, int variant) { return patch_rows(stages, variant) - 2 * stages; }
int patch_variants() { return kTileVariants; }

cudaError_t launch_step_patch_batch(const StepLaunch<float>& L, const BatchItem* items, int nitems,
                                    const BatchRep* reps, int variant) {
    const PatchArgs a = patch_args_common(L);
    const bool prec = L.precession != 0;
    if (L.tab->stages == 4)
        return batch_dispatch<4>(a, items, nitems, reps, L.stream, prec, L.pulse != 0, false, variant);
    return batch_dispatch<2>(a, items, nitems, reps, L.stream, prec, L.pulse != 0, false, variant);
}

cudaError_t prepare_patch_kernels() {
    {
        PatchArgs a{};
        cudaError_t e = batch_dispatch<4>(a, nullptr, 0, nullptr, 0, false, false, true, 0);
        if (e != cudaSuccess) return e;
        e = batch_dispatch<2>(a, nullptr, 0, nullptr, 0, false, false, true, 0);
        if (e != cudaSuccess) return e;
    }
    PatchArgs a{};
    cudaError_t e = patch_dispatch<4>(a, dim3(1), 0, false, false, false, true);
    if (e != cudaSuccess) return e;
    e = patch_dispatch<2>(a, dim3(1), 0, false, false, false, true);
    if (e != cudaSuccess) return e;
    e = patch_store_dispatch<4>(a, dim3(1), 0, false, false, true);
    if (e != cudaSuccess) return e;
    return patch_store_dispatch<2>(a, dim3(1), 0, false, false, true);
}

cudaError_t launch_step_patch(const StepLaunch<float>& L) {
    const int S = L.tab->stages;
    PatchArgs a = patch_args_common(L);
    const int outx = kPC - 2 * S;
    const int outy = patch_out_y(S, 0);
    const int tiles_x = (L.g.nx + outx - 1) / outx;
    const int tiles_y = (L.g.ny + outy - 1) / outy;
    // z chunks: one resident CTA per SM, so pick the chunk count that
    // minimises waves x (chunk planes + pipeline fill of 2S-2 iterations)
    const long long tiles = (long long)tiles_x * tiles_y;
    int best_chunks = 1;
    double best_cost = 1e300;
    for (int c = 1; c <= std::max(1, L.g.nz / 4); ++c) {
        const int zc_c = (L.g.nz + c - 1) / c;
        const int used = (L.g.nz + zc_c - 1) / zc_c;
        const long long ctas = tiles * used;
        const double waves = (double)((ctas + 151) / 152);
        const double cost = waves * (zc_c + 2 * S - 2);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best_chunks = c;
        }
    }
    const int zc = (L.g.nz + best_chunks - 1) / best_chunks;
    a.tz = zc;
    a.n_iter = zc + 2 * S - 2;
    dim3 grid(tiles_x, tiles_y, (L.g.nz + zc - 1) / zc);
    const bool hs = L.hs[0] != nullptr;
    const bool prec = L.precession != 0;
    cudaError_t e;
    if (L.st_n[0][0]) {
        for (int c = 0; c < 3; ++c) {
            for (int j = 0; j < S; ++j) {
                a.stn[j][c] = L.st_n[j][c];
                if (j + 1 < S) a.stx[j][c] = L.st_x[j][c];
            }
            a.sty[c] = L.st_y[c];
        }
        a.dt = (float)L.dt;
        e = S == 4 ? patch_store_dispatch<4>(a, grid, L.stream, prec, hs, false)
                   : patch_store_dispatch<2>(a, grid, L.stream, prec, hs, false);
    } else {
        e = S == 4 ? patch_dispatch<4>(a, grid, L.stream, prec, hs, false, false)
                   : patch_dispatch<2>(a, grid, L.stream, prec, hs, false, false);
    }
    if (e != cudaSuccess || !L.pulse) return e;
    return launch_pulse_lattice(L);
}

cudaError_t launch_pulse_lattice(const StepLaunch<float>& L) {
    const long long N = L.g.N();
    const int blocks = (int)std::max<long long>(1, std::min<long long>((N + 255) / 256, 152LL * 8));
    k_pulse_f32<<<blocks, 256, 0, L.stream>>>(L.out[0], L.out[1], L.out[2], N, L.seed, L.d_interval, L.replica,
                                              L.sigma);
    return cudaGetLastError();
}

}  // namespace spin
