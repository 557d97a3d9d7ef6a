// Device side of the fused FP32 z-marching step for chain tableaus (RK4,
// RK2 midpoint, Heun): tile geometry, register rings and one wavefront
// iteration, shared by the single-lattice kernels and the batched replicas.
//
// Geometry.  A CTA of 16 x TY threads owns a 32-column x (PY*TY)-row tile of
// lattice columns (x, y); each thread owns the column pair cx = 2tx, 2tx+1
// (one float2, so every FP32 operation of the right-hand side covers two
// sites with one f32x2 instruction) in PY rows.  The tile carries a halo of S
// columns and rows (S = stages): after stage j only the columns within S-j of
// the output block are still exact, which is all the next stage needs.  The
// CTA marches along z: at wavefront iteration t it streams in spin plane t+S
// and evaluates stage j on plane t+S-j, so every stage state lives on chip
// for exactly the planes its z-neighbours need (per-thread register rings
// indexed by plane & 3).
//
// Neighbour exchange per stage: x-neighbours by warp shuffles inside each
// 16-lane row segment, y-neighbours through shared memory (one double-
// buffered plane per stage, one barrier per iteration), z-neighbours from
// the rings.  One HBM read and one write of the state per step.
//
// Spin planes are staged in shared memory two iterations ahead, by per-thread
// cp.async copies of each thread's own column pair, or (optionally, RK4 on a
// single lattice whose sides are multiples of 4) by tensor-map bulk copies
// (TMA) of the tile in nine pieces, completion counted on an mbarrier per
// staging slot.
#pragma once
#include <cuda.h>
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
    int stg_off[PY];   // TMA staging: offset of the thread's column pair in a component's pieces
    bool bad;          // TMA staging: a bounded wait gave up (later waits are skipped)
};

// ---- TMA staging (RK4 tiles of 32 columns x ROWS rows, halo 4)
//
// A staged plane is cut into nine pieces per component: x widths 4 | 24 | 4
// and y heights 4 | ROWS-8 | 4.  With the lattice sides multiples of 4, at
// least 24 columns and ROWS-8 rows, and the last tile of each axis moved back
// so that its output block ends at the lattice edge, every piece lies wholly
// inside the lattice or wholly in its next periodic image: one TMA copy per
// piece at the wrapped origin (an x coordinate that is a multiple of 4 floats,
// so every copy starts on a 16-byte boundary).  Pieces are stored one after
// the other, each at a 128-byte boundary.  Tensor maps: per component, one
// map for each of the four piece shapes (4|24 wide x 4|ROWS-8 high).
struct TmaMaps {
    CUtensorMap m[3][4];   // [component][(width 24 ? 1 : 0) + (height ROWS-8 ? 2 : 0)]
};
__host__ __device__ constexpr int tma_w(int px) { return px == 1 ? 24 : 4; }
__host__ __device__ constexpr int tma_x0(int px) { return px == 0 ? 0 : (px == 1 ? 4 : 28); }
template <int ROWS>
__host__ __device__ constexpr int tma_h(int py) { return py == 1 ? ROWS - 8 : 4; }
template <int ROWS>
__host__ __device__ constexpr int tma_y0(int py) { return py == 0 ? 0 : (py == 1 ? 4 : ROWS - 4); }
__host__ __device__ constexpr int tma_pad(int n) { return (n + 31) & ~31; }
// offset (floats) of piece (py, px) within one component's pieces; piece 9 = end
template <int ROWS>
__host__ __device__ constexpr int tma_off(int piece) {
    int o = 0;
    for (int q = 0; q < piece; ++q) o += tma_pad(tma_w(q % 3) * tma_h<ROWS>(q / 3));
    return o;
}
template <int ROWS>
struct TmaSlot {
    static constexpr int COMP = tma_off<ROWS>(9);   // floats per component
    static constexpr int SLOT = 3 * COMP;           // floats per staging slot
    static constexpr unsigned BYTES = 3u * kPC * ROWS * 4u;   // bytes a staged plane brings
};

// Warp 0 stages the plane of wrapped z gz into slot q: lane 0 posts the byte
// count on the slot's mbarrier, then lanes 0..26 each issue one piece
// (component l/9, piece l%9).  The tile is (blockIdx.x, blockIdx.y) of the
// single-lattice grid, its origin recomputed here (the last tile of an axis
// moved back to end at the lattice edge), so no register holds it.
template <int ROWS>
__device__ __forceinline__ unsigned long long* tma_bars(float* stg) {
    return reinterpret_cast<unsigned long long*>(stg + 4 * TmaSlot<ROWS>::SLOT);
}
template <int ROWS>
__device__ __forceinline__ void tma_issue_plane(const TmaMaps* maps, float* stg, int q, int gz, int nx, int ny,
                                                int lane) {
    unsigned long long* bars = tma_bars<ROWS>(stg);
    constexpr int OUTX = kPC - 8, OUTY = ROWS - 8;
    const int ox = min((int)blockIdx.x * OUTX, nx - OUTX) - 4;
    const int oy = min((int)blockIdx.y * OUTY, ny - OUTY) - 4;
    if (lane == 0) mbar_arrive_expect_tx(bars + q, TmaSlot<ROWS>::BYTES);
    __syncwarp();
    if (lane < 27) {
        const int c = lane / 9, piece = lane % 9, px = piece % 3, py = piece / 3;
        int gx = ox + tma_x0(px), gy = oy + tma_y0<ROWS>(py);
        if (gx < 0) gx += nx;
        if (gx >= nx) gx -= nx;
        if (gy < 0) gy += ny;
        if (gy >= ny) gy -= ny;
        const CUtensorMap* m = &maps->m[c][(px == 1 ? 1 : 0) + (py == 1 ? 2 : 0)];
        float* dst = stg + q * TmaSlot<ROWS>::SLOT + c * TmaSlot<ROWS>::COMP + tma_off<ROWS>(piece);
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];\n" ::"r"(smem_addr(dst)),
            "l"(reinterpret_cast<unsigned long long>(m)), "r"(gx), "r"(gy), "r"(gz), "r"(smem_addr(bars + q))
            : "memory");
    }
}

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

// TMA staging context of a tile (unused by the cp.async staging)
struct TmaCtx {
    const TmaMaps* maps;   // tensor maps in the kernel's parameter space
};

template <int S, bool PREC, bool HSITE, bool PULSE, bool STORE, int P, int V, bool TMA>
__device__ __forceinline__ void patch_iteration(const PatchArgs& a, PRings<S, HSITE>& r, float* __restrict__ sh,
                                                float* __restrict__ stg, PThread<PatchShape<S>::PY>& th, int i,
                                                int t0, int z0, long long k, int tid, const TmaCtx& tc) {
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
        const int slot = (P + S) & 3;
        if constexpr (TMA) {
            // local plane i+S+2 into slot (P+S+2)&3, whose last plane (i+S-2)
            // every thread read before the barrier of iteration i-2; plane i+S
            // is the slot's fill number i>>2
            if (th.warp_row == 0)
                tma_issue_plane<ROWS>(tc.maps, stg, (P + S + 2) & 3, th.gz_issue, a.nx, a.ny, tid & 31);
            th.gz_issue = th.gz_issue + 1 == a.nz ? 0 : th.gz_issue + 1;
            mbar_wait(tma_bars<ROWS>(stg) + slot, (unsigned)((i >> 2) & 1), a.err, th.bad);
            const float* src = stg + slot * TmaSlot<ROWS>::SLOT;
#pragma unroll
            for (int rr = 0; rr < PY; ++rr)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    r.s[slot][rr][c] = *reinterpret_cast<const f2*>(src + c * TmaSlot<ROWS>::COMP + th.stg_off[rr]);
        } else {
            issue_plane<S, V>(a, stg, th, (P + S + 2) & 3, th.gz_issue, tid);
            th.gz_issue = th.gz_issue + 1 == a.nz ? 0 : th.gz_issue + 1;
            cp_async_wait<2>();
#pragma unroll
            for (int rr = 0; rr < PY; ++rr)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    r.s[slot][rr][c] = *reinterpret_cast<const f2*>(stage_pair<S, V>(stg, slot, c, rr, tid));
        }
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
//
// With TMA staging (TMA = true, RK4 only) the last tile of each axis is moved
// back so that its output block ends at the lattice edge (every staged piece
// then lies in one periodic image of the lattice); the columns it shares with
// the tile before it are written by that tile only.  maps are then the
// tensor maps (kernel parameter space); the grid must be the single-lattice
// grid (tile = blockIdx.x, blockIdx.y).
template <int S, bool PREC, bool HSITE, bool PULSE, bool STORE, int V, bool TMA = false>
__device__ __forceinline__ void patch_tile(const PatchArgs& a, int bx, int by, int bz, float* __restrict__ sh,
                                           const TmaMaps* maps = nullptr) {
    constexpr int PY = PatchShape<S, V>::PY, ROWS = PatchShape<S, V>::PY * PatchShape<S, V>::TY;
    static_assert(!TMA || (S == 4 && PY == 1), "TMA staging is laid out for RK4 tiles of one row per thread");
    float* stg = sh + 2 * S * 3 * ROWS * kRS;
    const int tid = threadIdx.y * kPT + threadIdx.x;
    PThread<PY> th;
    th.tx = threadIdx.x;
    th.ty = threadIdx.y;
    th.bad = false;
    // two thread rows per warp; broadcast from lane 0 so that the compiler
    // knows the index (and every stage-activity test built on it) is
    // warp-uniform and branches without divergence handling
    th.warp_row = __shfl_sync(0xffffffffu, (int)((threadIdx.y * kPT + threadIdx.x) >> 5), 0);
    constexpr int OUTX = kPC - 2 * S, OUTY = ROWS - 2 * S;
    th.plane = a.nx * a.ny;
    const int bx0 = bx * OUTX, by0 = by * OUTY;   // first output column / row this tile writes
    const int ox = (TMA ? min(bx0, a.nx - OUTX) : bx0) - S, oy = (TMA ? min(by0, a.ny - OUTY) : by0) - S;
    const TmaCtx tc{maps};
#pragma unroll
    for (int rr = 0; rr < PY; ++rr) {
        const int cy = PY * th.ty + rr;
        const int gyu = oy + cy;
        const int gy = wrapi(gyu, a.ny);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int cx = 2 * th.tx + e;
            const int gxu = ox + cx;
            th.col[rr][e] = gy * a.nx + wrapi(gxu, a.nx);
            th.out[rr][e] = cx >= S && cx < kPC - S && cy >= S && cy < ROWS - S && gxu < a.nx && gyu < a.ny &&
                            gxu >= bx0 && gyu >= by0;
            const float in = (gxu >= 0 && gxu < a.nx && gyu >= 0 && gyu < a.ny) ? 1.f : 0.f;
            if (e == 0) th.cmask[rr].x = a.bc ? in : 1.f;
            else th.cmask[rr].y = a.bc ? in : 1.f;
        }
        if constexpr (TMA) {
            const int cx = 2 * th.tx;
            const int px = cx < 4 ? 0 : (cx < 28 ? 1 : 2);
            const int py = cy < 4 ? 0 : (cy < ROWS - 4 ? 1 : 2);
            th.stg_off[rr] = tma_off<ROWS>(py * 3 + px) + (cy - tma_y0<ROWS>(py)) * tma_w(px) + (cx - tma_x0(px));
        } else {
            th.stg_off[rr] = 0;
        }
    }
    if constexpr (TMA) {
        if (tid == 0) {
            for (int q = 0; q < 4; ++q) mbar_init(tma_bars<ROWS>(stg) + q, 1);
            mbar_init_fence();
        }
        __syncthreads();
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
    if constexpr (TMA) {
        if (th.warp_row == 0) {
            tma_issue_plane<ROWS>(maps, stg, S & 3, wrapi(t0 + S, a.nz), a.nx, a.ny, tid & 31);
            tma_issue_plane<ROWS>(maps, stg, (S + 1) & 3, wrapi(t0 + S + 1, a.nz), a.nx, a.ny, tid & 31);
        }
    } else {
        issue_plane<S, V>(a, stg, th, S & 3, wrapi(t0 + S, a.nz), tid);
        issue_plane<S, V>(a, stg, th, (S + 1) & 3, wrapi(t0 + S + 1, a.nz), tid);
    }
    th.gz_issue = wrapi(t0 + S + 2, a.nz);
    th.gz_field = wrapi(t0 + S - 1, a.nz);
    int i = 0;
    for (; i + 4 <= a.n_iter; i += 4) {
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 0, V, TMA>(a, r, sh, stg, th, i + 0, t0, z0, k, tid, tc);
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 1, V, TMA>(a, r, sh, stg, th, i + 1, t0, z0, k, tid, tc);
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 2, V, TMA>(a, r, sh, stg, th, i + 2, t0, z0, k, tid, tc);
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 3, V, TMA>(a, r, sh, stg, th, i + 3, t0, z0, k, tid, tc);
    }
    if (i < a.n_iter)
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 0, V, TMA>(a, r, sh, stg, th, i + 0, t0, z0, k, tid, tc);
    if (i + 1 < a.n_iter)
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 1, V, TMA>(a, r, sh, stg, th, i + 1, t0, z0, k, tid, tc);
    if (i + 2 < a.n_iter)
        patch_iteration<S, PREC, HSITE, PULSE, STORE, 2, V, TMA>(a, r, sh, stg, th, i + 2, t0, z0, k, tid, tc);
    if constexpr (TMA) {
        // no copy may land in shared memory after the tile is done: the two
        // planes prefetched by the last two iterations (fills n_iter and
        // n_iter+1 counted from plane S) are awaited by the issuing warp
        if (th.warp_row == 0) {
            const int n = a.n_iter;
            mbar_wait(tma_bars<ROWS>(stg) + ((n + S) & 3), (unsigned)((n >> 2) & 1), a.err, th.bad);
            th.bad = false;   // the second copy is awaited even if the first wait gave up
            mbar_wait(tma_bars<ROWS>(stg) + ((n + 1 + S) & 3), (unsigned)(((n + 1) >> 2) & 1), a.err, th.bad);
        }
    } else {
        cp_async_wait<0>();   // no copy may land in shared memory after the tile is done
    }
}

// Dynamic shared memory of the cp.async-staged kernels: the double-buffered
// stage exchange planes and the per-thread staging ring.
template <int S, bool PREC, bool HSITE, bool PULSE, int V = 0>
size_t patch_smem() {
    constexpr int ROWS = PatchShape<S, V>::PY * PatchShape<S, V>::TY, NT = kPT * PatchShape<S, V>::TY;
    return sizeof(float) * (2 * S * 3 * ROWS * kRS + 4 * 3 * PatchShape<S, V>::PY * 2 * NT);
}

// Kernel arguments common to every fused-step launch of a lattice step.
inline PatchArgs patch_args_common(const StepLaunch<float>& L) {
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

}  // namespace
}  // namespace spin
