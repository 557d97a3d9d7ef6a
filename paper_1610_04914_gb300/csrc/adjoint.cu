// Discrete adjoint of the pulse-noise step (pathwise, noise fixed) for losses
// of the final state L = dLdE E(s_n) + dLdM . M(s_n), with checkpointing:
// the forward run stores the state every K steps; the backward pass restores
// each checkpoint, recomputes its K states with the forward kernels, and runs
// the transposed step backwards through them.  Parameter gradients (J, D, H,
// per-site h_i) accumulate in FP64: each site's term of each stage is formed
// in the state precision (like the forward stencil) and added in FP64, into
// the caller's FP64 field-gradient array (h_i) or into FP64 per-thread sums
// that are reduced in FP64 (J, D, H).
//
// Transposes used (f the right-hand side of Eq. LLL at fixed noise, a = s x H):
//   w_i = (df_i/dH_i)^T v_i = -(s x v) - lambda s x (s x v)    [slow: without -(s x v)]
//   u_i = (df_i/ds_i)^T v_i = H x v - lambda a x v + lambda H x (s x v)  [slow: without H x v]
//   (J_f^T v)_i = u_i + J sum_nn w_j + 2D w_iz z
//   renormalisation y -> y/|y|:  lam_y = (lam - u (u.lam))/|y|, u = y/|y|
//   pulse rotation R (Eq. s_rotation): lam <- R^T lam (rotation by -phi)
//   RK stages: lam_K_j = b_j lam_y, then for j = S..1: lam_x_j = J_f(x_j)^T (dt lam_K_j),
//              lam_s += lam_x_j, lam_K_l += a_jl lam_x_j (l < j)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "spin_device.cuh"
#include "spin_internal.h"

namespace spin {

namespace {

constexpr int kAT = 256;

// Neighbour indices x-1, x+1, y-1, y+1, z-1, z+1 (periodic wrap) of site i,
// and in w the weight of each: 0 for a neighbour across a face of a
// free-boundary lattice.  Two integer divisions per site, the wrap by
// comparison.
template <typename real>
__device__ __forceinline__ void neighbours_w(long long i, int nx, int ny, int nz, int bc, long long nb[6], real w[6]) {
    const int ii = (int)i;   // N < 2^31
    const int r = ii / nx;
    const int x = ii - r * nx;
    const int z = r / ny;
    const int y = r - z * ny;
    const long long P = (long long)nx * ny;
    const long long N = P * nz;
    nb[0] = x > 0 ? i - 1 : i + (nx - 1);
    nb[1] = x < nx - 1 ? i + 1 : i - (nx - 1);
    nb[2] = y > 0 ? i - nx : i + (long long)(ny - 1) * nx;
    nb[3] = y < ny - 1 ? i + nx : i - (long long)(ny - 1) * nx;
    nb[4] = z > 0 ? i - P : i + (N - P);
    nb[5] = z < nz - 1 ? i + P : i - (N - P);
    w[0] = (bc && x == 0) ? real(0) : real(1);
    w[1] = (bc && x == nx - 1) ? real(0) : real(1);
    w[2] = (bc && y == 0) ? real(0) : real(1);
    w[3] = (bc && y == ny - 1) ? real(0) : real(1);
    w[4] = (bc && z == 0) ? real(0) : real(1);
    w[5] = (bc && z == nz - 1) ? real(0) : real(1);
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

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

// H_eff at site i of a component-major 3N array x (FP32 or FP64 storage,
// evaluated in the storage precision like the forward kernels).
template <typename real, bool HSITE>
__device__ __forceinline__ void heff_at(const real* __restrict__ x, const real* __restrict__ hs, long long i,
                                        const long long nb[6], const real wn[6], long long N, real J, real twoD,
                                        const real H[3], real h[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const real* q = x + c * N;
        const real sum = wn[0] * q[nb[0]] + wn[1] * q[nb[1]] + wn[2] * q[nb[2]] + wn[3] * q[nb[3]] + wn[4] * q[nb[4]] +
                         wn[5] * q[nb[5]];
        h[c] = J * sum + H[c];
        if (HSITE) h[c] += hs[c * N + i];
    }
    h[2] += twoD * x[2 * N + i];
}

// K = dt f(x) over component-major arrays.
// Launch bounds for the stencil kernels of the backward pass: they are bound
// by the latency of the neighbour gathers, so four resident blocks per SM
// (at most 64 registers per thread) keep more loads in flight.
constexpr int kAdjMinBlocks = 4;

template <typename real, bool PREC, bool HSITE>
__global__ void __launch_bounds__(kAT, kAdjMinBlocks) k_adj_rhs(const real* __restrict__ x, const real* __restrict__ hs, real* __restrict__ K, int nx, int ny,
                          int nz, real J, real twoD, real H0, real H1, real H2, real lambda, real dt, int bc) {
    const long long N = (long long)nx * ny * nz;
    const real H[3] = {H0, H1, H2};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        long long nb[6];
        real wn[6];
        neighbours_w<real>(i, nx, ny, nz, bc, nb, wn);
        real h[3];
        heff_at<real, HSITE>(x, hs, i, nb, wn, N, J, twoD, H, h);
        real f[3];
        llg_rhs<real, PREC>(x[i], x[N + i], x[2 * N + i], h[0], h[1], h[2], lambda, f[0], f[1], f[2]);
        K[i] = dt * f[0];
        K[N + i] = dt * f[1];
        K[2 * N + i] = dt * f[2];
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

// Stage transpose, site-local part ("w-part") at site i for the stage with
// input x and v = dt lam_K: w and u, the per-site field gradient gh += w (in
// FP64), and the site's terms of <w, sum_nn x> (J), 2 x_z w_z (D) and w (H)
// added in FP64 to the thread's sums p[5].
template <typename real, bool PREC, bool HSITE>
__device__ __forceinline__ void w_part(const real* __restrict__ x, const real* __restrict__ hs, long long i,
                                       const long long nb[6], const real wn[6], long long N, real J, real twoD,
                                       const real H[3], real lambda, const real v[3], real* __restrict__ w,
                                       real* __restrict__ u, double* __restrict__ gh, double p[5]) {
    const real s[3] = {x[i], x[N + i], x[2 * N + i]};
    real sn[3], hr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const real* q = x + c * N;
        sn[c] = wn[0] * q[nb[0]] + wn[1] * q[nb[1]] + wn[2] * q[nb[2]] + wn[3] * q[nb[3]] + wn[4] * q[nb[4]] +
                wn[5] * q[nb[5]];
        hr[c] = J * sn[c] + H[c];
        if (HSITE) hr[c] += hs[c * N + i];
    }
    hr[2] += twoD * s[2];
    // the transpose in the state precision (like the forward stages)
    real a[3], sv[3], ssv[3], hv[3], av[3], hsv[3];
    cross3r(s, hr, a);
    cross3r(s, v, sv);
    cross3r(s, sv, ssv);
    cross3r(hr, v, hv);
    cross3r(a, v, av);
    cross3r(hr, sv, hsv);
    real wi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        real ui;
        if (PREC) {
            wi[c] = -sv[c] - lambda * ssv[c];
            ui = hv[c] - lambda * av[c] + lambda * hsv[c];
        } else {
            wi[c] = -lambda * ssv[c];
            ui = -lambda * av[c] + lambda * hsv[c];
        }
        w[c * N + i] = wi[c];
        u[c * N + i] = ui;
        if (gh) gh[c * N + i] += (double)wi[c];
    }
    p[0] += (double)(wi[0] * sn[0] + wi[1] * sn[1] + wi[2] * sn[2]);
    p[1] += (double)(real(2) * s[2] * wi[2]);
    p[2] += (double)wi[0];
    p[3] += (double)wi[1];
    p[4] += (double)wi[2];
}

// Block partials of the w-parts: the threads' FP64 sums are reduced in FP64
// (warp shuffles, then the block's warps in a fixed order) and added into the
// block's record.  Each block adds into its own record, launch after launch in
// stream order (deterministic); the records are summed once after the
// backward pass.
__device__ __forceinline__ void flush_partials(double p[5], double* __restrict__ partials) {
    __shared__ double red[kAT / 32][5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p[q] += __shfl_xor_sync(0xffffffffu, p[q], o);
    }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int q = 0; q < 5; ++q) red[threadIdx.x >> 5][q] = p[q];
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k][threadIdx.x];
        partials[(long long)blockIdx.x * 5 + threadIdx.x] += t;
    }
}

// Geometry and physics shared by the backward kernels.
template <typename real>
struct AdjGeom {
    int nx, ny, nz, bc;
    real J, twoD, H[3], lambda, dt;
};

// Top of the transposed step: pulse and renormalisation transposes, lam_s =
// lam_y, lam_K_j = b_j lam_y (stored for j < S-1), then the w-part of the
// last stage S-1, whose lam_K is not changed by any other stage.
template <typename real>
struct TopArgs {
    real* lam;           // in: dL/ds_after; out: lam_s = lam_y
    const real* s;       // state before the step
    LinComb<real> yc;    // y = s + sum_j b_j K_j, the unnormalised RK result
    real* LK[6];
    real b[6];
    int renorm, pulse;
    uint64_t seed, replica;
    long long k;
    real sigma;
    const real* xlast;   // input of stage S-1
    const real* hs;
    real* w;             // w, u of stage S-1
    real* u;
    double* gh;          // FP64 field gradient (3N) or null
    double* partials;
};

template <typename real, bool PREC, bool HSITE, int S>
__global__ void __launch_bounds__(kAT, kAdjMinBlocks) k_adj_top_w(TopArgs<real> a, AdjGeom<real> G) {
    const long long N = (long long)G.nx * G.ny * G.nz;
    double p[5] = {0, 0, 0, 0, 0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        real l0 = a.lam[i], l1 = a.lam[N + i], l2 = a.lam[2 * N + i];
        if (a.pulse) {
            const Words4 w = noise_words(a.seed, (uint64_t)i, (uint64_t)a.k, a.replica);
            real g0, g1, g2;
            Gauss<real>::draw(w, g0, g1, g2);
            pulse_rotate<real>(l0, l1, l2, -a.sigma * g0, -a.sigma * g1, -a.sigma * g2);
        }
        if (a.renorm) {
            const real y0 = lincomb_at<real, S>(a.s, a.yc, i), y1 = lincomb_at<real, S>(a.s, a.yc, N + i),
                       y2 = lincomb_at<real, S>(a.s, a.yc, 2 * N + i);
            const real n = Math<real>::sqrt_(y0 * y0 + y1 * y1 + y2 * y2);
            const real u0 = y0 / n, u1 = y1 / n, u2 = y2 / n;
            const real ul = u0 * l0 + u1 * l1 + u2 * l2;
            l0 = (l0 - u0 * ul) / n;
            l1 = (l1 - u1 * ul) / n;
            l2 = (l2 - u2 * ul) / n;
        }
        a.lam[i] = l0;
        a.lam[N + i] = l1;
        a.lam[2 * N + i] = l2;
#pragma unroll
        for (int j = 0; j < S - 1; ++j) {
            a.LK[j][i] = a.b[j] * l0;
            a.LK[j][N + i] = a.b[j] * l1;
            a.LK[j][2 * N + i] = a.b[j] * l2;
        }
        long long nb[6];
        real wn[6];
        neighbours_w<real>(i, G.nx, G.ny, G.nz, G.bc, nb, wn);
        const real bl = a.b[S - 1] * G.dt;
        const real v[3] = {bl * l0, bl * l1, bl * l2};
        w_part<real, PREC, HSITE>(a.xlast, a.hs, i, nb, wn, N, G.J, G.twoD, G.H, G.lambda, v, a.w, a.u, a.gh, p);
    }
    flush_partials(p, a.partials);
}

// Stage j of the transposed step: the neighbour part ("x-part") of stage j,
// lx = u_j + J sum_nn w_j + 2D w_jz z, lam_s += lx, lam_K_l += a_jl lx (l < j),
// and then (W) the w-part of stage j-1, which needs lam_K_{j-1} only at the
// same site and is final once stage j's x-part has added to it.  w and u of
// stage j are read from one buffer pair, those of stage j-1 written to the
// other.
template <typename real>
struct XWArgs {
    const real* w;       // stage j
    const real* u;
    real* lam;
    real* LK[6];
    real a[6];           // a_jl
    const real* xprev;   // input of stage j-1
    const real* hs;
    real* wn;            // w, u of stage j-1
    real* un;
    double* gh;          // FP64 field gradient (3N) or null
    double* partials;
};

template <typename real, bool PREC, bool HSITE, int NL, bool W>
__global__ void __launch_bounds__(kAT, kAdjMinBlocks) k_adj_xw(XWArgs<real> a, AdjGeom<real> G) {
    const long long N = (long long)G.nx * G.ny * G.nz;
    double p[5] = {0, 0, 0, 0, 0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        long long nb[6];
        real wn[6];
        neighbours_w<real>(i, G.nx, G.ny, G.nz, G.bc, nb, wn);
        real lk[3] = {0, 0, 0};   // lam_K_{j-1} at the site after this stage
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const real* q = a.w + c * N;
            real lx = a.u[c * N + i] + G.J * (wn[0] * q[nb[0]] + wn[1] * q[nb[1]] + wn[2] * q[nb[2]] +
                                              wn[3] * q[nb[3]] + wn[4] * q[nb[4]] + wn[5] * q[nb[5]]);
            if (c == 2) lx += G.twoD * a.w[2 * N + i];
            a.lam[c * N + i] += lx;
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                if (a.a[l] != real(0)) {
                    const real nv = a.LK[l][c * N + i] + a.a[l] * lx;
                    a.LK[l][c * N + i] = nv;
                    if (l == NL - 1) lk[c] = nv;
                } else if (l == NL - 1) {
                    lk[c] = a.LK[l][c * N + i];
                }
            }
        }
        if (W) {
            const real v[3] = {G.dt * lk[0], G.dt * lk[1], G.dt * lk[2]};
            w_part<real, PREC, HSITE>(a.xprev, a.hs, i, nb, wn, N, G.J, G.twoD, G.H, G.lambda, v, a.wn, a.un,
                                      a.gh, p);
        }
    }
    if (W) flush_partials(p, a.partials);
}

// acc[q] += sum over blocks of partials[b*5+q], fixed order (deterministic).
__global__ void k_adj_accumulate(const double* __restrict__ partials, int nblocks, double* __restrict__ acc, double scale) {
    __shared__ double red[kAT / 32];
    for (int q = 0; q < 5; ++q) {
        double v = 0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(long long)b * 5 + q];
        const double t = block_sum<double>(v, red);
        if (threadIdx.x == 0) acc[q] += scale * t;
    }
}

// Loss seed: lam_i = (-dLdE H_eff,i + dLdM)/N from the final state, with the
// explicit final-time terms: partials of bonds, sum s_z^2, M; gh += -dLdE s_i/N.
template <typename real, bool HSITE>
__global__ void __launch_bounds__(kAT) k_adj_seed(const real* __restrict__ s, const real* __restrict__ hs,
                                                  real* __restrict__ lam, double* __restrict__ gh,
                                                  double* __restrict__ partials, int nx, int ny, int nz, real J,
                                                  real twoD, real H0, real H1, real H2, double dLdE, double dM0,
                                                  double dM1, double dM2, int bc) {
    __shared__ double red[kAT / 32];
    const long long N = (long long)nx * ny * nz;
    const real H[3] = {H0, H1, H2};
    const double dM[3] = {dM0, dM1, dM2};
    double bonds = 0, sz2 = 0, m0 = 0, m1 = 0, m2 = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        long long nb[6];
        real wn[6];
        neighbours_w<real>(i, nx, ny, nz, bc, nb, wn);
        real h[3];
        heff_at<real, HSITE>(s, hs, i, nb, wn, N, J, twoD, H, h);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lam[c * N + i] = (real)((-dLdE * (double)h[c] + dM[c]) / (double)N);
            if (gh) gh[c * N + i] += -dLdE * (double)s[c * N + i] / (double)N;
        }
        const double a = s[i], b = s[N + i], c = s[2 * N + i];
        const double w1 = wn[1], w3 = wn[3], w5 = wn[5];   // forward bonds inside the lattice
        bonds += a * (w1 * s[nb[1]] + w3 * s[nb[3]] + w5 * s[nb[5]]) +
                 b * (w1 * s[N + nb[1]] + w3 * s[N + nb[3]] + w5 * s[N + nb[5]]) +
                 c * (w1 * s[2 * N + nb[1]] + w3 * s[2 * N + nb[3]] + w5 * s[2 * N + nb[5]]);
        sz2 += c * c;
        m0 += a;
        m1 += b;
        m2 += c;
    }
    const double vals[5] = {bonds, sz2, m0, m1, m2};
    for (int q = 0; q < 5; ++q) {
        const double t = block_sum<double>(vals[q], red);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * 5 + q] = t;
    }
}

// explicit terms -> gradient accumulators: acc = (gJ, gD, gH0, gH1, gH2)
__global__ void k_adj_seed_finish(const double* __restrict__ partials, int nblocks, double* __restrict__ acc, double dLdE,
                                  double N) {
    __shared__ double red[kAT / 32];
    double t[5];
    for (int q = 0; q < 5; ++q) {
        double v = 0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(long long)b * 5 + q];
        t[q] = block_sum<double>(v, red);
    }
    if (threadIdx.x == 0) {
        acc[0] += -dLdE * t[0] / N;
        acc[1] += -dLdE * t[1] / N;
        acc[2] += -dLdE * t[2] / N;
        acc[3] += -dLdE * t[3] / N;
        acc[4] += -dLdE * t[4] / N;
    }
}

template <typename real>
__global__ void k_gather3(real* __restrict__ dst, const real* __restrict__ s0, const real* __restrict__ s1,
                          const real* __restrict__ s2, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        dst[i] = s0[i];
        dst[N + i] = s1[i];
        dst[2 * N + i] = s2[i];
    }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + kAT - 1) / kAT, 152LL * 8)); }

}  // namespace

int adjoint_blocks(Geom g) { return grid_for(g.N()); }

constexpr size_t kStageStoreMax = (size_t)8 << 30;   // bytes of stage storage at most

bool adjoint_stores_stages(const Geom& g, int elt, const Tableau& tb, int path, int K) {
    if (elt != 4 || !tb.chain || path == 1 || !(tb.stages == 2 || tb.stages == 4)) return false;
    const size_t comp = ((size_t)3 * (size_t)g.N() * 4 + 255) / 256 * 256;
    return comp * (size_t)(2 * tb.stages - 1) * (size_t)K <= kStageStoreMax;
}

size_t adjoint_workspace_bytes(const Geom& g, int elt, const Tableau& tb, int path, int K) {
    const int stages = tb.stages;
    const size_t comp = (size_t)3 * (size_t)g.N() * (size_t)elt;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    size_t b = 0;
    if (adjoint_stores_stages(g, elt, tb, path, K))
        b += al(comp) * (size_t)(2 * stages - 1) * (size_t)K;   // X_j (j >= 2) and K_j of every step of a segment
    b += al(comp) * (size_t)(K + 1);     // segment states
    b += al(comp) * (size_t)stages * 3;  // X_j, K_j, lam_K_j
    b += al(comp) * 6;                   // y, lam, w and u (two pairs)
    b += al(sizeof(double) * 5 * (size_t)adjoint_blocks(g));
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

template <typename real, bool PREC, bool HSITE>
void launch_xw_t(int j, const XWArgs<real>& a, const AdjGeom<real>& G, int gb, cudaStream_t st) {
    switch (j) {
        case 0: k_adj_xw<real, PREC, HSITE, 0, false><<<gb, kAT, 0, st>>>(a, G); break;
        case 1: k_adj_xw<real, PREC, HSITE, 1, true><<<gb, kAT, 0, st>>>(a, G); break;
        case 2: k_adj_xw<real, PREC, HSITE, 2, true><<<gb, kAT, 0, st>>>(a, G); break;
        case 3: k_adj_xw<real, PREC, HSITE, 3, true><<<gb, kAT, 0, st>>>(a, G); break;
        case 4: k_adj_xw<real, PREC, HSITE, 4, true><<<gb, kAT, 0, st>>>(a, G); break;
        default: k_adj_xw<real, PREC, HSITE, 5, true><<<gb, kAT, 0, st>>>(a, G); break;
    }
}

// x-part of stage j and (j > 0) w-part of stage j-1.
template <typename real>
void launch_xw(bool prec, bool hsite, int j, const XWArgs<real>& a, const AdjGeom<real>& G, int gb, cudaStream_t st) {
    if (prec) {
        if (hsite) launch_xw_t<real, true, true>(j, a, G, gb, st);
        else launch_xw_t<real, true, false>(j, a, G, gb, st);
    } else {
        if (hsite) launch_xw_t<real, false, true>(j, a, G, gb, st);
        else launch_xw_t<real, false, false>(j, a, G, gb, st);
    }
}

template <typename real, bool PREC, bool HSITE>
void launch_top_w_t(int S, const TopArgs<real>& a, const AdjGeom<real>& G, int gb, cudaStream_t st) {
    if (S == 2) k_adj_top_w<real, PREC, HSITE, 2><<<gb, kAT, 0, st>>>(a, G);
    else if (S == 4) k_adj_top_w<real, PREC, HSITE, 4><<<gb, kAT, 0, st>>>(a, G);
    else k_adj_top_w<real, PREC, HSITE, 6><<<gb, kAT, 0, st>>>(a, G);
}

template <typename real>
void launch_top_w(bool prec, bool hsite, int S, const TopArgs<real>& a, const AdjGeom<real>& G, int gb,
                  cudaStream_t st) {
    if (prec) {
        if (hsite) launch_top_w_t<real, true, true>(S, a, G, gb, st);
        else launch_top_w_t<real, true, false>(S, a, G, gb, st);
    } else {
        if (hsite) launch_top_w_t<real, false, true>(S, a, G, gb, st);
        else launch_top_w_t<real, false, false>(S, a, G, gb, st);
    }
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
    real* y = reinterpret_cast<real*>(ws + off);
    off += al(compb);
    real* lam = reinterpret_cast<real*>(ws + off);
    off += al(compb);
    real* wb[2];   // w and u of the stages, double-buffered by stage parity
    real* ub[2];
    for (int q = 0; q < 2; ++q) {
        wb[q] = reinterpret_cast<real*>(ws + off);
        off += al(compb);
        ub[q] = reinterpret_cast<real*>(ws + off);
        off += al(compb);
    }
    const int nb = adjoint_blocks(g);
    double* partials = reinterpret_cast<double*>(ws + off);
    off += al(sizeof(double) * 5 * (size_t)nb);
    double* acc = reinterpret_cast<double*>(ws + off);
    off += al(sizeof(double) * 8);
    long long* kslot = reinterpret_cast<long long*>(ws + off);
    off += al(sizeof(long long));
    // stage storage of a segment (A.store_stages): for step m of the segment
    // (slot m-1) the inputs X_2..X_S and the increments K_1..K_S
    const bool stored = A.store_stages != 0;
    char* sbase = ws + off;
    auto stage_x = [&](int j, int m) {   // X_j, j = 2..S (0-based stage index j-1 >= 1)
        return reinterpret_cast<real*>(sbase + ((size_t)(m - 1) * (2 * S - 1) + (size_t)(j - 2)) * al(compb));
    };
    auto stage_k = [&](int j, int m) {   // K_j, j = 1..S
        return reinterpret_cast<real*>(sbase + ((size_t)(m - 1) * (2 * S - 1) + (size_t)(S - 1) + (size_t)(j - 1)) * al(compb));
    };
    cudaStream_t st = A.stream;
    const real J = (real)A.J, twoD = (real)(2.0 * A.D), H0 = (real)A.H[0], H1 = (real)A.H[1], H2 = (real)A.H[2];
    const real lamb = (real)A.lambda, dt = (real)A.dt;
    const real* hs = A.h_site;
    const bool HS = hs != nullptr;
    AdjGeom<real> G{};
    G.nx = g.nx;
    G.ny = g.ny;
    G.nz = g.nz;
    G.bc = A.bc;
    G.J = J;
    G.twoD = twoD;
    G.H[0] = H0;
    G.H[1] = H1;
    G.H[2] = H2;
    G.lambda = lamb;
    G.dt = dt;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 8, st);
    if (e != cudaSuccess) return e;

    // seed from the final state (component arrays of the caller)
    real* fin = y;  // temporarily gather the final state
    k_gather3<real><<<grid_for(N), kAT, 0, st>>>(fin, A.final_state[0], A.final_state[1], A.final_state[2], N);
    if (HS)
        k_adj_seed<real, true><<<nb, kAT, 0, st>>>(fin, hs, lam, A.g_h, partials, g.nx, g.ny, g.nz, J, twoD, H0, H1, H2,
                                                   A.dLdE, A.dLdM[0], A.dLdM[1], A.dLdM[2], A.bc);
    else
        k_adj_seed<real, false><<<nb, kAT, 0, st>>>(fin, nullptr, lam, A.g_h, partials, g.nx, g.ny, g.nz, J, twoD, H0, H1,
                                                    H2, A.dLdE, A.dLdM[0], A.dLdM[1], A.dLdM[2], A.bc);
    k_adj_seed_finish<<<1, kAT, 0, st>>>(partials, nb, acc, A.dLdE, (double)N);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // per-block FP64 records of the stage transposes start at zero
    e = cudaMemsetAsync(partials, 0, sizeof(double) * 5 * (size_t)nb, st);
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
                for (int j = 1; j <= S; ++j)
                    for (int c = 0; c < 3; ++c) {
                        L.st_k[j - 1][c] = stage_k(j, m) + c * N;
                        if (j >= 2) L.st_x[j - 2][c] = stage_x(j, m) + c * N;
                    }
            }
            e = launch_step<real>(L);
            if (e != cudaSuccess) return e;
        }
        // transposed steps, last to first
        for (int m = seglen; m >= 1; --m) {
            const long long n = start + m;
            const bool pul = A.noise && (n % A.R) == (A.R / 2);
            const real* s = seg + (size_t)(m - 1) * len;
            // stages X_j and K_j = dt f(X_j); the first stage's input is s itself
            const real* Xs[6];
            real* Kp[6];
            for (int j = 0; j < S; ++j) Kp[j] = stored ? stage_k(j + 1, m) : Kst[j];
            for (int j = 0; j < S && stored; ++j) Xs[j] = j == 0 ? s : stage_x(j + 1, m);
            for (int j = 0; j < S && !stored; ++j) {
                if (j == 0) {
                    Xs[0] = s;
                } else {
                    LinComb<real> lc{};
                    for (int l = 0; l < j; ++l) {
                        lc.K[l] = Kst[l];
                        lc.coef[l] = (real)tb.a[j][l];
                    }
                    launch_lincomb<real>(j, X[j], s, lc, len, st);
                    Xs[j] = X[j];
                }
                if (A.precession) {
                    if (HS) k_adj_rhs<real, true, true><<<grid_for(N), kAT, 0, st>>>(Xs[j], hs, Kst[j], g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                    else k_adj_rhs<real, true, false><<<grid_for(N), kAT, 0, st>>>(Xs[j], nullptr, Kst[j], g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                } else {
                    if (HS) k_adj_rhs<real, false, true><<<grid_for(N), kAT, 0, st>>>(Xs[j], hs, Kst[j], g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                    else k_adj_rhs<real, false, false><<<grid_for(N), kAT, 0, st>>>(Xs[j], nullptr, Kst[j], g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                }
            }
            TopArgs<real> ta{};
            ta.lam = lam;
            ta.s = s;
            for (int l = 0; l < S; ++l) {
                ta.yc.K[l] = Kp[l];
                ta.yc.coef[l] = (real)tb.b[l];
            }
            for (int j = 0; j < S; ++j) {
                ta.LK[j] = LK[j];
                ta.b[j] = (real)tb.b[j];
            }
            ta.renorm = A.renorm;
            ta.pulse = pul ? 1 : 0;
            ta.seed = A.seed;
            ta.replica = A.replica;
            ta.k = (n - 1) / A.R;
            ta.sigma = (real)A.sigma;
            ta.xlast = Xs[S - 1];
            ta.hs = hs;
            ta.w = wb[(S - 1) & 1];
            ta.u = ub[(S - 1) & 1];
            ta.gh = A.g_h;
            ta.partials = partials;
            launch_top_w<real>(A.precession != 0, HS, S, ta, G, nb, st);
            for (int j = S - 1; j >= 0; --j) {
                XWArgs<real> xa{};
                xa.w = wb[j & 1];
                xa.u = ub[j & 1];
                xa.lam = lam;
                for (int l = 0; l < j; ++l) {
                    xa.LK[l] = LK[l];
                    xa.a[l] = (real)tb.a[j][l];
                }
                if (j > 0) {
                    xa.xprev = Xs[j - 1];
                    xa.wn = wb[(j - 1) & 1];
                    xa.un = ub[(j - 1) & 1];
                }
                xa.hs = hs;
                xa.gh = A.g_h;
                xa.partials = partials;
                launch_xw<real>(A.precession != 0, HS, j, xa, G, nb, st);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    k_adj_accumulate<<<1, kAT, 0, st>>>(partials, nb, acc, 1.0);
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
