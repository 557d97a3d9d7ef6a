// Discrete adjoint of the pulse-noise step (pathwise, noise fixed) for losses
// of the final state L = dLdE E(s_n) + dLdM . M(s_n), with checkpointing:
// the forward run stores the state every K steps; the backward pass restores
// each checkpoint, recomputes its K states with the forward kernels, and runs
// the transposed step backwards through them.
//
// Parameter gradients accumulate in FP64: every site's term of every stage is
// formed in the state precision (like the forward stencil) and added in FP64
// into per-site FP64 arrays -- dL/dh_i (3N), and the site's dL/dJ and dL/dD
// terms (N each), which are summed over the sites in FP64 once, after the
// backward pass.  H enters the effective field exactly as every h_i
// does, so dL/dH = sum_i dL/dh_i is that array's FP64 sum (explicit final-time
// term included).  The float-to-double conversions of the terms are done with
// integer bit operations (exact for every finite float), because this GPU's
// FP64 pipe, which would otherwise convert them, is ~1/76 of its FP32 rate.
//
// Transposes used (f the right-hand side of Eq. LLL at fixed noise, a = s x H):
//   w_i = (df_i/dH_i)^T v_i = -(s x v) - lambda s x (s x v)    [slow: without -(s x v)]
//   u_i = (df_i/ds_i)^T v_i = H x v - lambda a x v + lambda H x (s x v)  [slow: without H x v]
//   (J_f^T v)_i = u_i + J sum_nn w_j + 2D w_iz z
//   renormalisation y -> y/|y|:  lam_y = (lam - u (u.lam))/|y|, u = y/|y|
//   pulse rotation R (Eq. s_rotation): lam <- R^T lam (rotation by -phi)
//   RK stages: lam_K_j = b_j lam_y, then for j = S..1: lam_x_j = J_f(x_j)^T (dt lam_K_j),
//              lam_s += lam_x_j, lam_K_l += a_jl lam_x_j (l < j)
//
// Indexing: a 3D grid of (row segment of 32 x-sites, group of 8 rows, plane),
// one thread per site and one warp per row segment, so no coordinate needs a
// division; every array is addressed through per-component base pointers with
// 32-bit site offsets.  For FP32 chain tableaus the recomputing forward step
// stores, per step of a segment, the stage inputs X_j (j >= 2), the stage
// neighbour sums sum_nn X_j (j >= 1) and the unnormalised RK result y; the
// transposes then read them instead of recomputing any stencil of X_j.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "spin_device.cuh"
#include "spin_internal.h"

namespace spin {

namespace {

constexpr int kAT = 256;                 // threads per block (8 warps)
constexpr int kAW = kAT / 32;

// Programmatic dependent launch of the transposed-step kernels: each is
// launched while the kernel before it drains, and waits (griddepcontrol.wait,
// a no-op without a programmatic dependency) for that kernel's completion and
// memory before touching global memory; each lets its successor launch once
// all of its blocks have stored their results.
// Resident blocks per SM asked of the chain-tableau transposes: 6 blocks of
// 256 threads cap them at 40 registers (from 44-48), so a 64^3 lattice's 1024
// blocks take 1.12 rounds of 152 SMs instead of 1.35; measured 4.5% faster
// per backward step with the programmatic-dependent launches (8 blocks, 32
// registers: 1%).
#ifndef SPIN_ADJ_MINB
#define SPIN_ADJ_MINB 6
#endif
#ifndef SPIN_ADJ_PDL
#define SPIN_ADJ_PDL 1
#endif
__device__ __forceinline__ void pdl_wait() {
#if SPIN_ADJ_PDL
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_trigger() {
#if SPIN_ADJ_PDL
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
#endif
}
template <typename Kern, typename... Args>
cudaError_t pdl_launch(Kern kernel, dim3 grid, cudaStream_t st, Args... args) {
#if SPIN_ADJ_PDL
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kAT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
#else
    kernel<<<grid, kAT, 0, st>>>(args...);
    return cudaGetLastError();
#endif
}

// A site of the lattice with its six neighbours (x-1, x+1, y-1, y+1, z-1, z+1;
// periodic wrap) and their weights (0 across a face of a free-boundary
// lattice).  All indices fit in 32 bits (N < 2^31).
template <typename real>
struct Site {
    int i;
    int nb[6];
    real wn[6];
    bool valid;
};

// The site of this thread: the 3D grid is (row segment of 32 x-sites, group of
// 8 rows, plane), one warp per row segment, so no coordinate needs a division.
template <typename real>
__device__ __forceinline__ Site<real> site_here(int nx, int ny, int nz, int bc) {
    Site<real> s;
    const int x = (int)(blockIdx.x * 32 + (threadIdx.x & 31));
    const int y0 = (int)(blockIdx.y * kAW + (threadIdx.x >> 5));
    const int z = (int)blockIdx.z;
    s.valid = x < nx && y0 < ny;
    const int xx = x < nx ? x : nx - 1;        // idle lanes read a valid site and write nothing
    const int y = y0 < ny ? y0 : ny - 1;
    const int P = nx * ny;
    const int i = (z * ny + y) * nx + xx;
    s.i = i;
    s.nb[0] = xx > 0 ? i - 1 : i + (nx - 1);
    s.nb[1] = xx < nx - 1 ? i + 1 : i - (nx - 1);
    s.nb[2] = y > 0 ? i - nx : i + (ny - 1) * nx;
    s.nb[3] = y < ny - 1 ? i + nx : i - (ny - 1) * nx;
    s.nb[4] = z > 0 ? i - P : i + (nz - 1) * P;
    s.nb[5] = z < nz - 1 ? i + P : i - (nz - 1) * P;
    s.wn[0] = (bc && xx == 0) ? real(0) : real(1);
    s.wn[1] = (bc && xx == nx - 1) ? real(0) : real(1);
    s.wn[2] = (bc && y == 0) ? real(0) : real(1);
    s.wn[3] = (bc && y == ny - 1) ? real(0) : real(1);
    s.wn[4] = (bc && z == 0) ? real(0) : real(1);
    s.wn[5] = (bc && z == nz - 1) ? real(0) : real(1);
    return s;
}

// Record of this block in the per-block partial sums.
__device__ __forceinline__ int block_record() {
    return (int)(blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
}

// Component arrays (x, y, z blocks of a 3N array).
template <typename real>
struct V3 {
    real* c[3];
};
template <typename real>
struct CV3 {
    const real* c[3];
};

template <typename real>
__device__ __forceinline__ void cross3r(const real a[3], const real b[3], real c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    return t;
}

// Geometry and physics shared by the backward kernels.
template <typename real>
struct AdjGeom {
    int nx, ny, nz, bc;
    long long N;
    real J, twoD, H[3], lambda, dt;
};

// Neighbour sum of one component array at a site.
template <typename real>
__device__ __forceinline__ real nbsum(const real* __restrict__ q, const Site<real>& st) {
    return st.wn[0] * q[st.nb[0]] + st.wn[1] * q[st.nb[1]] + st.wn[2] * q[st.nb[2]] + st.wn[3] * q[st.nb[3]] +
           st.wn[4] * q[st.nb[4]] + st.wn[5] * q[st.nb[5]];
}

// K = dt f(x) over component arrays (stages recomputed in the backward pass
// when they are not stored).
template <typename real, bool PREC, bool HSITE>
__global__ void __launch_bounds__(kAT) k_adj_rhs(CV3<real> x, CV3<real> hs, V3<real> K, AdjGeom<real> G) {
    const Site<real> st = site_here<real>(G.nx, G.ny, G.nz, G.bc);
    const int i = st.i;
    real h[3], s[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s[c] = x.c[c][i];
        h[c] = G.J * nbsum<real>(x.c[c], st) + G.H[c];
        if (HSITE) h[c] += hs.c[c][i];
    }
    h[2] += G.twoD * s[2];
    real f[3];
    llg_rhs<real, PREC>(s[0], s[1], s[2], h[0], h[1], h[2], G.lambda, f[0], f[1], f[2]);
    if (st.valid) {
#pragma unroll
        for (int c = 0; c < 3; ++c) K.c[c][i] = G.dt * f[c];
    }
}

// out = s + sum_l coef[l] K_l: a stage input, or the RK combination y.  The
// number of terms is a template argument (dispatched once on the host), so
// the pointer table is indexed with constants and stays in kernel parameters.
template <typename real>
struct LinComb {
    const real* K[6];
    real coef[6];
};

template <typename real, int NK>
__device__ __forceinline__ real lincomb_at(const real* __restrict__ s, const LinComb<real>& lc, long long q) {
    real acc = s[q];
#pragma unroll
    for (int l = 0; l < NK; ++l) acc += lc.coef[l] * lc.K[l][q];
    return acc;
}

template <typename real, int NK>
__global__ void k_adj_lincomb(real* __restrict__ out, const real* __restrict__ s, LinComb<real> lc, long long len) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < len; q += (long long)gridDim.x * blockDim.x)
        out[q] = lincomb_at<real, NK>(s, lc, q);
}

// Inputs of a stage's w-part: its input x and the neighbour sum of x (stored,
// or computed here from x when sn.c[0] is null).
template <typename real>
struct StageIn {
    CV3<real> x, sn;
};

// Stage transpose, site-local part ("w-part") at a site for the stage with
// input x and v = dt lam_K: w and u, the per-site field gradient gh += w (FP64)
// and the site's terms <w, sum_nn x> (J) and 2 x_z w_z (D) added in FP64 to
// the site's entries of gjd (J at i, D at N + i).  (One FP64 add per term and
// site: on this GPU's narrow FP64 pipe a per-block tree reduction, at five
// adds per warp and value, measured slower.)
// Every load of the site is issued before the arithmetic.
template <typename real, bool PREC, bool HSITE>
__device__ __forceinline__ void w_part(const StageIn<real>& in, const CV3<real>& hs, const Site<real>& st,
                                       const AdjGeom<real>& G, const real v[3], const V3<real>& w, const V3<real>& u,
                                       const V3<double>& gh, double* __restrict__ gjd) {
    const int i = st.i;
    real s[3], sn[3], hsv[3];
    double g[3];
    const double gj = gjd[i], gd = gjd[G.N + i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s[c] = in.x.c[c][i];
        sn[c] = in.sn.c[0] ? in.sn.c[c][i] : nbsum<real>(in.x.c[c], st);
        hsv[c] = HSITE ? hs.c[c][i] : real(0);
        g[c] = gh.c[c][i];
    }
    real hr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        hr[c] = G.J * sn[c] + G.H[c];
        if (HSITE) hr[c] += hsv[c];
    }
    hr[2] += G.twoD * s[2];
    // the transpose in the state precision (like the forward stages)
    real a[3], sv[3], ssv[3], hv[3], av[3], hsx[3];
    cross3r(s, hr, a);
    cross3r(s, v, sv);
    cross3r(s, sv, ssv);
    cross3r(hr, v, hv);
    cross3r(a, v, av);
    cross3r(hr, sv, hsx);
    real wi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        real ui;
        if (PREC) {
            wi[c] = -sv[c] - G.lambda * ssv[c];
            ui = hv[c] - G.lambda * av[c] + G.lambda * hsx[c];
        } else {
            wi[c] = -G.lambda * ssv[c];
            ui = -G.lambda * av[c] + G.lambda * hsx[c];
        }
        if (!st.valid) wi[c] = real(0);
        if (st.valid) {
            w.c[c][i] = wi[c];
            u.c[c][i] = ui;
            gh.c[c][i] = g[c] + to_f64(wi[c]);
        }
    }
    if (st.valid) {
        gjd[i] = gj + to_f64(wi[0] * sn[0] + wi[1] * sn[1] + wi[2] * sn[2]);
        gjd[G.N + i] = gd + to_f64(real(2) * s[2] * wi[2]);
    }
}

// Top of the transposed step: pulse and renormalisation transposes, lam_s =
// lam_y, lam_K_j = b_j lam_y (stored for j < S-1; for chain tableaus lam_y
// itself is stored instead, since there lam_K_j = b_j lam_y + a_{j+1,j} lx_{j+1}
// is formed where it is used), then the w-part of the
// last stage S-1, whose lam_K is not changed by any other stage.
template <typename real>
struct TopArgs {
    V3<real> lam;        // in: dL/ds_after; out: lam_s = lam_y
    const real* s;       // state before the step (3N)
    CV3<real> ystored;   // the unnormalised RK result, when the step stored it (c[0] null otherwise)
    LinComb<real> yc;    // otherwise y = s + sum_j b_j K_j (3N arrays)
    V3<real> LK[6];
    V3<real> ly;         // chain tableaus: lam_y
    real b[6];
    int renorm, pulse;
    uint64_t seed, replica;
    long long k;
    real sigma;
    StageIn<real> last;  // input of stage S-1 and its neighbour sum
    CV3<real> hs;
    V3<real> w, u;       // w, u of stage S-1
    V3<double> gh;       // FP64 field gradient
    double* gjd;         // FP64 per-site dL/dJ (N) and dL/dD (N) terms
};

// The top at a site, given the adjoint (l0, l1, l2) of the step's output.
template <typename real, bool PREC, bool HSITE, int S, bool CHAIN>
__device__ __forceinline__ void top_body(const TopArgs<real>& a, const AdjGeom<real>& G, const Site<real>& st, real l0,
                                         real l1, real l2) {
    const int i = st.i;
    if (a.pulse) {
        const Words4 wd = noise_words(a.seed, (uint64_t)i, (uint64_t)a.k, a.replica);
        real g0, g1, g2;
        Gauss<real>::draw(wd, g0, g1, g2);
        pulse_rotate<real>(l0, l1, l2, -a.sigma * g0, -a.sigma * g1, -a.sigma * g2);
    }
    if (a.renorm) {
        real y0, y1, y2;
        if (a.ystored.c[0]) {
            y0 = a.ystored.c[0][i];
            y1 = a.ystored.c[1][i];
            y2 = a.ystored.c[2][i];
        } else {
            y0 = lincomb_at<real, S>(a.s, a.yc, i);
            y1 = lincomb_at<real, S>(a.s, a.yc, G.N + i);
            y2 = lincomb_at<real, S>(a.s, a.yc, 2 * G.N + i);
        }
        const real n = Math<real>::sqrt_(y0 * y0 + y1 * y1 + y2 * y2);
        const real u0 = y0 / n, u1 = y1 / n, u2 = y2 / n;
        const real ul = u0 * l0 + u1 * l1 + u2 * l2;
        l0 = (l0 - u0 * ul) / n;
        l1 = (l1 - u1 * ul) / n;
        l2 = (l2 - u2 * ul) / n;
    }
    if (st.valid) {
        a.lam.c[0][i] = l0;
        a.lam.c[1][i] = l1;
        a.lam.c[2][i] = l2;
        if (CHAIN) {
            a.ly.c[0][i] = l0;
            a.ly.c[1][i] = l1;
            a.ly.c[2][i] = l2;
        } else {
#pragma unroll
            for (int j = 0; j < S - 1; ++j) {
                a.LK[j].c[0][i] = a.b[j] * l0;
                a.LK[j].c[1][i] = a.b[j] * l1;
                a.LK[j].c[2][i] = a.b[j] * l2;
            }
        }
    }
    const real bl = a.b[S - 1] * G.dt;
    const real v[3] = {bl * l0, bl * l1, bl * l2};
    w_part<real, PREC, HSITE>(a.last, a.hs, st, G, v, a.w, a.u, a.gh, a.gjd);
}

template <typename real, bool PREC, bool HSITE, int S, bool CHAIN>
__global__ void __launch_bounds__(kAT) k_adj_top_w(TopArgs<real> a, AdjGeom<real> G) {
    pdl_wait();
    const Site<real> st = site_here<real>(G.nx, G.ny, G.nz, G.bc);
    const int i = st.i;
    top_body<real, PREC, HSITE, S, CHAIN>(a, G, st, a.lam.c[0][i], a.lam.c[1][i], a.lam.c[2][i]);
    pdl_trigger();
}

// Stage j of the transposed step: the neighbour part ("x-part") of stage j,
// lx = u_j + J sum_nn w_j + 2D w_jz z, lam_s += lx, lam_K_l += a_jl lx (l < j),
// and then (W) the w-part of stage j-1, which needs lam_K_{j-1} only at the
// same site and is final once stage j's x-part has added to it.  For chain
// tableaus lam_K_{j-1} = b_{j-1} lam_y + a_{j,j-1} lx is formed here from
// lam_y (no lam_K arrays).  w and u of stage j are read from one buffer pair,
// those of stage j-1 written to the other.
template <typename real>
struct XWArgs {
    CV3<real> w, u;      // stage j
    V3<real> lam;
    V3<real> LK[6];
    CV3<real> ly;        // chain tableaus: lam_y
    real a[6];           // a_jl
    real bl;             // chain tableaus: b_{j-1}
    StageIn<real> prev;  // input of stage j-1 and its neighbour sum
    CV3<real> hs;
    V3<real> wn, un;     // w, u of stage j-1
    V3<double> gh;       // FP64 field gradient
    double* gjd;         // FP64 per-site dL/dJ (N) and dL/dD (N) terms
};

template <typename real, bool PREC, bool HSITE, int NL, bool W, bool CHAIN>
__global__ void __launch_bounds__(kAT, CHAIN ? SPIN_ADJ_MINB : 1) k_adj_xw(XWArgs<real> a, AdjGeom<real> G) {
    pdl_wait();
    const Site<real> st = site_here<real>(G.nx, G.ny, G.nz, G.bc);
    const int i = st.i;
    constexpr int NLOAD = CHAIN ? 1 : (NL > 0 ? NL : 1);
    real ux[3], lm[3], wz, nsum[3], lkv[NLOAD][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ux[c] = a.u.c[c][i];
        lm[c] = a.lam.c[c][i];
        nsum[c] = nbsum<real>(a.w.c[c], st);
        if (CHAIN) {
            if (NL > 0) lkv[0][c] = a.ly.c[c][i];
        } else {
#pragma unroll
            for (int l = 0; l < NL; ++l) lkv[l][c] = a.LK[l].c[c][i];
        }
    }
    wz = a.w.c[2][i];
    real lk[3] = {0, 0, 0};   // lam_K_{j-1} at the site after this stage
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        real lx = ux[c] + G.J * nsum[c];
        if (c == 2) lx += G.twoD * wz;
        if (st.valid) a.lam.c[c][i] = lm[c] + lx;
        if (CHAIN) {
            if (NL > 0) {
                const real base = a.bl * lkv[0][c];
                lk[c] = base + a.a[NL - 1] * lx;
            }
        } else {
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                if (a.a[l] != real(0)) {
                    const real nv = lkv[l][c] + a.a[l] * lx;
                    if (st.valid) a.LK[l].c[c][i] = nv;
                    if (l == NL - 1) lk[c] = nv;
                } else if (l == NL - 1) {
                    lk[c] = lkv[l][c];
                }
            }
        }
    }
    if (W) {
        const real v[3] = {G.dt * lk[0], G.dt * lk[1], G.dt * lk[2]};
        w_part<real, PREC, HSITE>(a.prev, a.hs, st, G, v, a.wn, a.un, a.gh, a.gjd);
    }
    pdl_trigger();
}

// The first stage's x-part of step m (lam_s += lx, final: the adjoint of step
// m's input state) fused with the top of step m-1, which needs that adjoint
// at the same site only: one launch and one read and write of lam fewer per
// step.  For steps whose stages were stored (the top then reads only stored
// arrays of step m-1).
template <typename real, bool PREC, bool HSITE, int S, bool CHAIN>
__global__ void __launch_bounds__(kAT, CHAIN ? SPIN_ADJ_MINB : 1) k_adj_x0_top(XWArgs<real> a, TopArgs<real> ta, AdjGeom<real> G) {
    pdl_wait();
    const Site<real> st = site_here<real>(G.nx, G.ny, G.nz, G.bc);
    const int i = st.i;
    real ux[3], lm[3], nsum[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ux[c] = a.u.c[c][i];
        lm[c] = a.lam.c[c][i];
        nsum[c] = nbsum<real>(a.w.c[c], st);
    }
    const real wz = a.w.c[2][i];
    real l[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        real lx = ux[c] + G.J * nsum[c];
        if (c == 2) lx += G.twoD * wz;
        l[c] = lm[c] + lx;
    }
    top_body<real, PREC, HSITE, S, CHAIN>(ta, G, st, l[0], l[1], l[2]);
    pdl_trigger();
}

// FP64 sums of kSumParts consecutive parts of each of the arrays at v + c N
// (c < gridDim.y, N doubles each): block (p, c) writes parts[c kSumParts + p];
// fixed order (deterministic).
constexpr int kSumParts = 152;
__global__ void k_adj_sum_parts(const double* __restrict__ v, long long N, double* __restrict__ parts) {
    __shared__ double red[kAW];
    const long long c = blockIdx.y, p = blockIdx.x;
    const long long lo = p * N / kSumParts, hi = (p + 1) * N / kSumParts;
    const double* g = v + c * N;
    double t = 0;
    for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x) t += g[q];
    t = block_sum<double>(t, red);
    if (threadIdx.x == 0) parts[c * kSumParts + p] = t;
}

// acc[first + c] (+)= the FP64 sum of parts[c kSumParts ...] (one block per
// array, fixed order): dL/dJ, dL/dD (added to the seed's explicit terms) from
// the per-site terms, dL/dH = sum_i dL/dh_i from the field gradient.
__global__ void k_adj_sum_final(const double* __restrict__ parts, double* __restrict__ acc, int first, int add) {
    __shared__ double red[kAW];
    const double* g = parts + (long long)blockIdx.x * kSumParts;
    double v = 0;
    for (int q = threadIdx.x; q < kSumParts; q += blockDim.x) v += g[q];
    const double t = block_sum<double>(v, red);
    if (threadIdx.x == 0) acc[first + blockIdx.x] = add ? acc[first + blockIdx.x] + t : t;
}

// Loss seed: lam_i = (-dLdE H_eff,i + dLdM)/N from the final state, with the
// explicit final-time terms: partials of bonds (J) and sum s_z^2 (D);
// gh += -dLdE s_i/N (the explicit dE/dh_i, which also gives dE/dH through the
// final sum of gh).
template <typename real, bool HSITE>
__global__ void __launch_bounds__(kAT) k_adj_seed(CV3<real> s, CV3<real> hs, V3<real> lam, V3<double> gh,
                                                  double* __restrict__ partials, AdjGeom<real> G, double dLdE,
                                                  double dM0, double dM1, double dM2) {
    __shared__ double red[kAW];
    const long long N = G.N;
    const double dM[3] = {dM0, dM1, dM2};
    double bonds = 0, sz2 = 0;
    const Site<real> st = site_here<real>(G.nx, G.ny, G.nz, G.bc);
    const int i = st.i;
    real h[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        h[c] = G.J * nbsum<real>(s.c[c], st) + G.H[c];
        if (HSITE) h[c] += hs.c[c][i];
    }
    h[2] += G.twoD * s.c[2][i];
    if (st.valid) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lam.c[c][i] = (real)((-dLdE * (double)h[c] + dM[c]) / (double)N);
            gh.c[c][i] += -dLdE * (double)s.c[c][i] / (double)N;
        }
        const double a = s.c[0][i], b = s.c[1][i], c = s.c[2][i];
        const double w1 = st.wn[1], w3 = st.wn[3], w5 = st.wn[5];   // forward bonds inside the lattice
        const int* nb = st.nb;
        bonds = a * (w1 * s.c[0][nb[1]] + w3 * s.c[0][nb[3]] + w5 * s.c[0][nb[5]]) +
                b * (w1 * s.c[1][nb[1]] + w3 * s.c[1][nb[3]] + w5 * s.c[1][nb[5]]) +
                c * (w1 * s.c[2][nb[1]] + w3 * s.c[2][nb[3]] + w5 * s.c[2][nb[5]]);
        sz2 = c * c;
    }
    const double vals[2] = {bonds, sz2};
    for (int q = 0; q < 2; ++q) {
        const double t = block_sum<double>(vals[q], red);
        if (threadIdx.x == 0) partials[(long long)block_record() * 2 + q] = t;
    }
}

// explicit terms -> gradient accumulators acc = (gJ, gD)
__global__ void k_adj_seed_finish(const double* __restrict__ partials, int nblocks, double* __restrict__ acc,
                                  double dLdE, double N) {
    __shared__ double red[kAW];
    double t[2];
    for (int q = 0; q < 2; ++q) {
        double v = 0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(long long)b * 2 + q];
        t[q] = block_sum<double>(v, red);
    }
    if (threadIdx.x == 0) {
        acc[0] += -dLdE * t[0] / N;
        acc[1] += -dLdE * t[1] / N;
    }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + kAT - 1) / kAT, 152LL * 8)); }

// The 3D grid of the site kernels: row segments of 32 x-sites, groups of 8
// rows (one per warp), planes.
dim3 grid3(const Geom& g) { return dim3((g.nx + 31) / 32, (g.ny + kAW - 1) / kAW, g.nz); }

}  // namespace

int adjoint_blocks(Geom g) {
    const dim3 d = grid3(g);
    return (int)(d.x * d.y * d.z);
}

constexpr size_t kStageStoreMax = (size_t)8 << 30;   // bytes of stage storage at most

// Stored per step of a segment: X_j (j = 2..S), sum_nn X_j (j = 1..S) and y:
// 2S arrays of 3N floats.
bool adjoint_stores_stages(const Geom& g, int elt, const Tableau& tb, int path, int K) {
    if (elt != 4 || !tb.chain || path == 1 || !(tb.stages == 2 || tb.stages == 4)) return false;
    const size_t comp = ((size_t)3 * (size_t)g.N() * 4 + 255) / 256 * 256;
    return comp * (size_t)(2 * tb.stages) * (size_t)K <= kStageStoreMax;
}

size_t adjoint_workspace_bytes(const Geom& g, int elt, const Tableau& tb, int path, int K) {
    const int stages = tb.stages;
    const size_t comp = (size_t)3 * (size_t)g.N() * (size_t)elt;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    size_t b = 0;
    if (adjoint_stores_stages(g, elt, tb, path, K))
        b += al(comp) * (size_t)(2 * stages) * (size_t)K;   // X_j, sum_nn X_j and y of every step of a segment
    b += al(comp) * (size_t)(K + 1);     // segment states
    b += al(comp) * (size_t)stages * 3;  // X_j, K_j, lam_K_j (lam_y in the first for chain tableaus)
    b += al(comp) * 6;                   // y, lam, w and u (two pairs)
    b += al(sizeof(double) * 3 * (size_t)g.N());   // FP64 field gradient when the caller does not want it
    b += al(sizeof(double) * 2 * (size_t)g.N());   // FP64 per-site dL/dJ and dL/dD terms
    b += al(sizeof(double) * 5 * (size_t)kSumParts);           // per-part sums of those and of the field gradient
    b += al(sizeof(double) * 2 * (size_t)adjoint_blocks(g));   // the seed's per-block partials
    b += al(sizeof(double) * 8);         // accumulators
    b += al(sizeof(long long));          // pulse-number slot
    return b;
}

// Launch the combine kernels with the term count as a template argument.
template <typename real>
void launch_lincomb(int nk, real* out, const real* s, const LinComb<real>& lc, long long len, cudaStream_t st) {
    const int gb = grid_for(len);
    switch (nk) {
        case 0: k_adj_lincomb<real, 0><<<gb, kAT, 0, st>>>(out, s, lc, len); break;
        case 1: k_adj_lincomb<real, 1><<<gb, kAT, 0, st>>>(out, s, lc, len); break;
        case 2: k_adj_lincomb<real, 2><<<gb, kAT, 0, st>>>(out, s, lc, len); break;
        case 3: k_adj_lincomb<real, 3><<<gb, kAT, 0, st>>>(out, s, lc, len); break;
        case 4: k_adj_lincomb<real, 4><<<gb, kAT, 0, st>>>(out, s, lc, len); break;
        default: k_adj_lincomb<real, 5><<<gb, kAT, 0, st>>>(out, s, lc, len); break;
    }
}

// The tableaus of the library: chain tableaus (RK4, RK2 midpoint, Heun) have
// 2 or 4 stages, Butcher's RK5 (6 stages) is not a chain.
inline bool adj_tableau_supported(int S, bool chain) { return chain ? (S == 2 || S == 4) : S == 6; }

template <typename real, bool PREC, bool HSITE>
cudaError_t launch_xw_t(int j, int S, bool chain, const XWArgs<real>& a, const AdjGeom<real>& G, dim3 gb,
                        cudaStream_t st) {
    if (!adj_tableau_supported(S, chain)) return cudaErrorInvalidValue;
    if (chain) {
        switch (j) {
            case 0: return pdl_launch(k_adj_xw<real, PREC, HSITE, 0, false, true>, gb, st, a, G);
            case 1: return pdl_launch(k_adj_xw<real, PREC, HSITE, 1, true, true>, gb, st, a, G);
            case 2: return pdl_launch(k_adj_xw<real, PREC, HSITE, 2, true, true>, gb, st, a, G);
            case 3: return pdl_launch(k_adj_xw<real, PREC, HSITE, 3, true, true>, gb, st, a, G);
            default: return cudaErrorInvalidValue;
        }
        return cudaSuccess;
    }
    switch (j) {
        case 0: return pdl_launch(k_adj_xw<real, PREC, HSITE, 0, false, false>, gb, st, a, G);
        case 1: return pdl_launch(k_adj_xw<real, PREC, HSITE, 1, true, false>, gb, st, a, G);
        case 2: return pdl_launch(k_adj_xw<real, PREC, HSITE, 2, true, false>, gb, st, a, G);
        case 3: return pdl_launch(k_adj_xw<real, PREC, HSITE, 3, true, false>, gb, st, a, G);
        case 4: return pdl_launch(k_adj_xw<real, PREC, HSITE, 4, true, false>, gb, st, a, G);
        case 5: return pdl_launch(k_adj_xw<real, PREC, HSITE, 5, true, false>, gb, st, a, G);
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

// x-part of stage j and (j > 0) w-part of stage j-1.
template <typename real>
cudaError_t launch_xw(bool prec, bool hsite, int j, int S, bool chain, const XWArgs<real>& a, const AdjGeom<real>& G,
                      dim3 gb, cudaStream_t st) {
    if (prec) {
        if (hsite) return launch_xw_t<real, true, true>(j, S, chain, a, G, gb, st);
        return launch_xw_t<real, true, false>(j, S, chain, a, G, gb, st);
    }
    if (hsite) return launch_xw_t<real, false, true>(j, S, chain, a, G, gb, st);
    return launch_xw_t<real, false, false>(j, S, chain, a, G, gb, st);
}

template <typename real, bool PREC, bool HSITE>
cudaError_t launch_x0_top_t(int S, bool chain, const XWArgs<real>& xa, const TopArgs<real>& ta, const AdjGeom<real>& G,
                            dim3 gb, cudaStream_t st) {
    if (chain && S == 2) return pdl_launch(k_adj_x0_top<real, PREC, HSITE, 2, true>, gb, st, xa, ta, G);
    else if (chain && S == 4) return pdl_launch(k_adj_x0_top<real, PREC, HSITE, 4, true>, gb, st, xa, ta, G);
    else return cudaErrorInvalidValue;
    return cudaSuccess;
}

template <typename real>
cudaError_t launch_x0_top(bool prec, bool hsite, int S, bool chain, const XWArgs<real>& xa, const TopArgs<real>& ta,
                          const AdjGeom<real>& G, dim3 gb, cudaStream_t st) {
    if (prec) {
        if (hsite) return launch_x0_top_t<real, true, true>(S, chain, xa, ta, G, gb, st);
        return launch_x0_top_t<real, true, false>(S, chain, xa, ta, G, gb, st);
    }
    if (hsite) return launch_x0_top_t<real, false, true>(S, chain, xa, ta, G, gb, st);
    return launch_x0_top_t<real, false, false>(S, chain, xa, ta, G, gb, st);
}

template <typename real, bool PREC, bool HSITE>
cudaError_t launch_top_w_t(int S, bool chain, const TopArgs<real>& a, const AdjGeom<real>& G, dim3 gb,
                           cudaStream_t st) {
    if (chain && S == 2) return pdl_launch(k_adj_top_w<real, PREC, HSITE, 2, true>, gb, st, a, G);
    else if (chain && S == 4) return pdl_launch(k_adj_top_w<real, PREC, HSITE, 4, true>, gb, st, a, G);
    else if (!chain && S == 6) return pdl_launch(k_adj_top_w<real, PREC, HSITE, 6, false>, gb, st, a, G);
    else return cudaErrorInvalidValue;
    return cudaSuccess;
}

template <typename real>
cudaError_t launch_top_w(bool prec, bool hsite, int S, bool chain, const TopArgs<real>& a, const AdjGeom<real>& G,
                         dim3 gb, cudaStream_t st) {
    if (prec) {
        if (hsite) return launch_top_w_t<real, true, true>(S, chain, a, G, gb, st);
        return launch_top_w_t<real, true, false>(S, chain, a, G, gb, st);
    }
    if (hsite) return launch_top_w_t<real, false, true>(S, chain, a, G, gb, st);
    return launch_top_w_t<real, false, false>(S, chain, a, G, gb, st);
}

template <typename real>
V3<real> v3(real* base, long long N) {
    V3<real> v;
    for (int c = 0; c < 3; ++c) v.c[c] = base ? base + c * N : nullptr;
    return v;
}
template <typename real>
CV3<real> cv3(const real* base, long long N) {
    CV3<real> v;
    for (int c = 0; c < 3; ++c) v.c[c] = base ? base + c * N : nullptr;
    return v;
}

template <typename real>
cudaError_t adjoint_run(const AdjointRun<real>& A) {
    const Geom g = A.g;
    const long long N = g.N(), len = 3 * N;
    const Tableau& tb = *A.tab;
    const int S = tb.stages;
    const size_t compb = (size_t)len * sizeof(real);
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    char* ws = static_cast<char*>(A.workspace);
    size_t off = 0;
    real* seg = reinterpret_cast<real*>(ws + off);
    off += al(compb) * (size_t)(A.K + 1);
    real* X[6];
    real* Kst[6];
    real* LK[6];
    for (int j = 0; j < S; ++j) {
        X[j] = reinterpret_cast<real*>(ws + off);
        off += al(compb);
    }
    for (int j = 0; j < S; ++j) {
        Kst[j] = reinterpret_cast<real*>(ws + off);
        off += al(compb);
    }
    for (int j = 0; j < S; ++j) {
        LK[j] = reinterpret_cast<real*>(ws + off);
        off += al(compb);
    }
    off += al(compb);   // (unused slot, kept so the layout matches adjoint_workspace_bytes)
    real* lam = reinterpret_cast<real*>(ws + off);
    off += al(compb);
    if (!adj_tableau_supported(S, tb.chain)) return cudaErrorInvalidValue;
    real* wb[2];   // w and u of the stages, double-buffered by stage parity
    real* ub[2];
    for (int q = 0; q < 2; ++q) {
        wb[q] = reinterpret_cast<real*>(ws + off);
        off += al(compb);
        ub[q] = reinterpret_cast<real*>(ws + off);
        off += al(compb);
    }
    // the FP64 field gradient: the caller's array, or a workspace one (dL/dH
    // is its sum either way)
    double* gh = A.g_h ? A.g_h : reinterpret_cast<double*>(ws + off);
    off += al(sizeof(double) * 3 * (size_t)N);
    const int nb = adjoint_blocks(g);
    const dim3 gb = grid3(g);
    double* gjd = reinterpret_cast<double*>(ws + off);
    off += al(sizeof(double) * 2 * (size_t)N);
    double* parts = reinterpret_cast<double*>(ws + off);
    off += al(sizeof(double) * 5 * (size_t)kSumParts);
    double* partials = reinterpret_cast<double*>(ws + off);
    off += al(sizeof(double) * 2 * (size_t)nb);
    double* acc = reinterpret_cast<double*>(ws + off);
    off += al(sizeof(double) * 8);
    long long* kslot = reinterpret_cast<long long*>(ws + off);
    off += al(sizeof(long long));
    // stage storage of a segment (A.store_stages): for step m of the segment
    // (slot m-1) the inputs X_2..X_S, the neighbour sums of X_1..X_S and y
    const bool stored = A.store_stages != 0;
    char* sbase = ws + off;
    auto slot_arr = [&](int m, int q) {
        return reinterpret_cast<real*>(sbase + ((size_t)(m - 1) * (2 * S) + (size_t)q) * al(compb));
    };
    auto stage_x = [&](int j, int m) { return slot_arr(m, j - 2); };           // X_j, j = 2..S
    auto stage_sn = [&](int j, int m) { return slot_arr(m, S - 1 + j - 1); };  // sum_nn X_j, j = 1..S
    auto stage_y = [&](int m) { return slot_arr(m, 2 * S - 1); };
    cudaStream_t st = A.stream;
    const real* hs = A.h_site;
    const bool HS = hs != nullptr;
    const CV3<real> hs3 = cv3<real>(hs, N);
    const V3<double> gh3 = v3<double>(gh, N);
    AdjGeom<real> G{};
    G.nx = g.nx;
    G.ny = g.ny;
    G.nz = g.nz;
    G.bc = A.bc;
    G.N = N;
    G.J = (real)A.J;
    G.twoD = (real)(2.0 * A.D);
    G.H[0] = (real)A.H[0];
    G.H[1] = (real)A.H[1];
    G.H[2] = (real)A.H[2];
    G.lambda = (real)A.lambda;
    G.dt = (real)A.dt;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 8, st);
    if (e != cudaSuccess) return e;
    if (!A.g_h && (e = cudaMemsetAsync(gh, 0, sizeof(double) * 3 * (size_t)N, st)) != cudaSuccess) return e;

    // seed from the final state (component arrays of the caller)
    CV3<real> fin;
    for (int c = 0; c < 3; ++c) fin.c[c] = A.final_state[c];
    if (HS)
        k_adj_seed<real, true><<<gb, kAT, 0, st>>>(fin, hs3, v3<real>(lam, N), gh3, partials, G, A.dLdE, A.dLdM[0],
                                                   A.dLdM[1], A.dLdM[2]);
    else
        k_adj_seed<real, false><<<gb, kAT, 0, st>>>(fin, hs3, v3<real>(lam, N), gh3, partials, G, A.dLdE, A.dLdM[0],
                                                    A.dLdM[1], A.dLdM[2]);
    k_adj_seed_finish<<<1, kAT, 0, st>>>(partials, nb, acc, A.dLdE, (double)N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the per-site FP64 J and D terms start at zero
    e = cudaMemsetAsync(gjd, 0, sizeof(double) * 2 * (size_t)N, st);
    if (e != cudaSuccess) return e;

    const long long total = A.n_end - A.n0;
    const int nseg = (int)((total + A.K - 1) / A.K);
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const long long start = A.n0 + (long long)sgi * A.K;
        const int seglen = (int)std::min<long long>(A.K, A.n_end - start);
        // restore checkpoint and recompute the segment with the forward kernels;
        // the transposed steps read the states 0 .. seglen-1 of the segment,
        // so its last state is not recomputed unless the steps also store
        // their stages (then every step of the segment runs)
        e = cudaMemcpyAsync(seg, A.store + (size_t)sgi * len, compb, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        for (int m = 1; m < seglen + (stored ? 1 : 0); ++m) {
            const long long n = start + m;
            const bool pul = A.noise && (n % A.R) == (A.R / 2);
            if (pul) {
                e = launch_set_counter(kslot, (n - 1) / A.R, st);
                if (e != cudaSuccess) return e;
            }
            StepLaunch<real> L = A.step_template;
            real* prev = seg + (size_t)(m - 1) * len;
            real* next = seg + (size_t)m * len;
            for (int c = 0; c < 3; ++c) {
                L.in[c] = prev + c * N;
                L.out[c] = next + c * N;
            }
            L.pulse = pul ? 1 : 0;
            L.d_interval = kslot;
            L.stream = st;
            if (stored) {
                for (int c = 0; c < 3; ++c) {
                    for (int j = 1; j <= S; ++j) {
                        L.st_n[j - 1][c] = stage_sn(j, m) + c * N;
                        if (j >= 2) L.st_x[j - 2][c] = stage_x(j, m) + c * N;
                    }
                    L.st_y[c] = stage_y(m) + c * N;
                }
            }
            e = launch_step<real>(L);
            if (e != cudaSuccess) return e;
        }
        // transposed steps, last to first.  With stored stages the first
        // stage's x-part of step m and the top of step m-1 share a launch.
        auto stage_inputs = [&](int m, StageIn<real>* in) {
            const real* s = seg + (size_t)(m - 1) * len;
            // the first stage's input is s itself
            for (int j = 0; j < S; ++j) {
                in[j].x = cv3<real>((j == 0) ? s : (stored ? stage_x(j + 1, m) : X[j]), N);
                in[j].sn = cv3<real>(stored ? stage_sn(j + 1, m) : nullptr, N);
            }
        };
        auto top_args = [&](int m, const StageIn<real>* in) {
            const long long n = start + m;
            const bool pul = A.noise && (n % A.R) == (A.R / 2);
            TopArgs<real> ta{};
            ta.lam = v3<real>(lam, N);
            ta.s = seg + (size_t)(m - 1) * len;
            ta.ystored = cv3<real>(stored ? stage_y(m) : nullptr, N);
            for (int l = 0; l < S; ++l) {
                ta.yc.K[l] = Kst[l];
                ta.yc.coef[l] = (real)tb.b[l];
            }
            for (int j = 0; j < S; ++j) {
                ta.LK[j] = v3<real>(LK[j], N);
                ta.b[j] = (real)tb.b[j];
            }
            ta.ly = v3<real>(LK[0], N);   // chain tableaus: lam_y in the first lam_K buffer
            ta.renorm = A.renorm;
            ta.pulse = pul ? 1 : 0;
            ta.seed = A.seed;
            ta.replica = A.replica;
            ta.k = (n - 1) / A.R;
            ta.sigma = (real)A.sigma;
            ta.last = in[S - 1];
            ta.hs = hs3;
            ta.w = v3<real>(wb[(S - 1) & 1], N);
            ta.u = v3<real>(ub[(S - 1) & 1], N);
            ta.gh = gh3;
            ta.gjd = gjd;
            return ta;
        };
        auto xw_args = [&](int j, const StageIn<real>* in) {
            XWArgs<real> xa{};
            xa.w = cv3<real>(wb[j & 1], N);
            xa.u = cv3<real>(ub[j & 1], N);
            xa.lam = v3<real>(lam, N);
            for (int l = 0; l < j; ++l) {
                xa.LK[l] = v3<real>(LK[l], N);
                xa.a[l] = (real)tb.a[j][l];
            }
            xa.ly = cv3<real>(LK[0], N);
            xa.bl = j > 0 ? (real)tb.b[j - 1] : real(0);
            if (j > 0) {
                xa.prev = in[j - 1];
                xa.wn = v3<real>(wb[(j - 1) & 1], N);
                xa.un = v3<real>(ub[(j - 1) & 1], N);
            }
            xa.hs = hs3;
            xa.gh = gh3;
            xa.gjd = gjd;
            return xa;
        };
        const bool fuse_top = stored && tb.chain;
        for (int m = seglen; m >= 1; --m) {
            const real* s = seg + (size_t)(m - 1) * len;
            StageIn<real> in[6];
            stage_inputs(m, in);
            // stages X_j and K_j = dt f(X_j), recomputed when not stored
            for (int j = 0; j < S && !stored; ++j) {
                if (j > 0) {
                    LinComb<real> lc{};
                    for (int l = 0; l < j; ++l) {
                        lc.K[l] = Kst[l];
                        lc.coef[l] = (real)tb.a[j][l];
                    }
                    launch_lincomb<real>(j, X[j], s, lc, len, st);
                }
                const V3<real> K3 = v3<real>(Kst[j], N);
                if (A.precession) {
                    if (HS) k_adj_rhs<real, true, true><<<gb, kAT, 0, st>>>(in[j].x, hs3, K3, G);
                    else k_adj_rhs<real, true, false><<<gb, kAT, 0, st>>>(in[j].x, hs3, K3, G);
                } else {
                    if (HS) k_adj_rhs<real, false, true><<<gb, kAT, 0, st>>>(in[j].x, hs3, K3, G);
                    else k_adj_rhs<real, false, false><<<gb, kAT, 0, st>>>(in[j].x, hs3, K3, G);
                }
            }
            if (!fuse_top || m == seglen) {
                const TopArgs<real> ta = top_args(m, in);
                if ((e = launch_top_w<real>(A.precession != 0, HS, S, tb.chain, ta, G, gb, st)) != cudaSuccess)
                    return e;
            }
            for (int j = S - 1; j >= 0; --j) {
                const XWArgs<real> xa = xw_args(j, in);
                if (j == 0 && fuse_top && m > 1) {
                    StageIn<real> inp[6];
                    stage_inputs(m - 1, inp);
                    const TopArgs<real> ta = top_args(m - 1, inp);
                    if ((e = launch_x0_top<real>(A.precession != 0, HS, S, tb.chain, xa, ta, G, gb, st)) != cudaSuccess)
                        return e;
                } else if ((e = launch_xw<real>(A.precession != 0, HS, j, S, tb.chain, xa, G, gb, st)) != cudaSuccess) {
                    return e;
                }
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    // dL/dJ, dL/dD (added to the seed's explicit terms) and dL/dH: FP64 sums in
    // two deterministic passes
    k_adj_sum_parts<<<dim3(kSumParts, 2), kAT, 0, st>>>(gjd, N, parts);
    k_adj_sum_parts<<<dim3(kSumParts, 3), kAT, 0, st>>>(gh, N, parts + 2 * kSumParts);
    k_adj_sum_final<<<2, kAT, 0, st>>>(parts, acc, 0, 1);
    k_adj_sum_final<<<3, kAT, 0, st>>>(parts + 2 * kSumParts, acc, 2, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // results: gradient accumulators to the host, dL/ds_0 to the caller
    if (A.g_s0) {
        e = cudaMemcpyAsync(A.g_s0, lam, compb, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    double host[5];
    e = cudaMemcpyAsync(host, acc, sizeof(host), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *A.gJ = host[0];
    *A.gD = host[1];
    A.gH[0] = host[2];
    A.gH[1] = host[3];
    A.gH[2] = host[4];
    return cudaSuccess;
}

template cudaError_t adjoint_run<float>(const AdjointRun<float>&);
template cudaError_t adjoint_run<double>(const AdjointRun<double>&);

}  // namespace spin
