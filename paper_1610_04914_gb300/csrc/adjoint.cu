// Discrete adjoint of the pulse-noise step (pathwise, noise fixed) for losses
// of the final state L = dLdE E(s_n) + dLdM . M(s_n), with checkpointing:
// the forward run stores the state every K steps; the backward pass restores
// each checkpoint, recomputes its K states with the forward kernels, and runs
// the transposed step backwards through them.  Parameter gradients (J, D, H,
// per-site h_i) accumulate in FP64.
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

__device__ __forceinline__ int wrapa(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ void site_xyz(long long i, int nx, int ny, int& x, int& y, int& z) {
    const int ii = (int)i;   // N < 2^31
    x = ii % nx;
    const int r = ii / nx;
    y = r % ny;
    z = r / ny;
}

// Neighbour indices x-1, x+1, y-1, y+1, z-1, z+1 (periodic), and in w the
// weight of each: 0 for a neighbour across a face of a free-boundary lattice.
template <typename real>
__device__ __forceinline__ void neighbour_weights(long long i, int nx, int ny, int nz, int bc, real w[6]) {
    int x, y, z;
    const int ii = (int)i;
    x = ii % nx;
    y = (ii / nx) % ny;
    z = (ii / nx) / ny;
    w[0] = (bc && x == 0) ? real(0) : real(1);
    w[1] = (bc && x == nx - 1) ? real(0) : real(1);
    w[2] = (bc && y == 0) ? real(0) : real(1);
    w[3] = (bc && y == ny - 1) ? real(0) : real(1);
    w[4] = (bc && z == 0) ? real(0) : real(1);
    w[5] = (bc && z == nz - 1) ? real(0) : real(1);
}

__device__ __forceinline__ void neighbours(long long i, int nx, int ny, int nz, long long nb[6]) {
    int x, y, z;
    site_xyz(i, nx, ny, x, y, z);
    const long long P = (long long)nx * ny;
    const long long row = (long long)z * P + (long long)y * nx;
    nb[0] = row + wrapa(x - 1, nx);
    nb[1] = row + wrapa(x + 1, nx);
    nb[2] = (long long)z * P + (long long)wrapa(y - 1, ny) * nx + x;
    nb[3] = (long long)z * P + (long long)wrapa(y + 1, ny) * nx + x;
    nb[4] = (long long)wrapa(z - 1, nz) * P + (long long)y * nx + x;
    nb[5] = (long long)wrapa(z + 1, nz) * P + (long long)y * nx + x;
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
template <typename real, bool PREC, bool HSITE>
__global__ void k_adj_rhs(const real* __restrict__ x, const real* __restrict__ hs, real* __restrict__ K, int nx, int ny,
                          int nz, real J, real twoD, real H0, real H1, real H2, real lambda, real dt, int bc) {
    const long long N = (long long)nx * ny * nz;
    const real H[3] = {H0, H1, H2};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        long long nb[6];
        neighbours(i, nx, ny, nz, nb);
        real wn[6];
        neighbour_weights<real>(i, nx, ny, nz, bc, wn);
        real h[3];
        heff_at<real, HSITE>(x, hs, i, nb, wn, N, J, twoD, H, h);
        real f[3];
        llg_rhs<real, PREC>(x[i], x[N + i], x[2 * N + i], h[0], h[1], h[2], lambda, f[0], f[1], f[2]);
        K[i] = dt * f[0];
        K[N + i] = dt * f[1];
        K[2 * N + i] = dt * f[2];
    }
}

// out = s + sum_l coef[l] K_l over 3N elements.
template <typename real>
struct LinComb {
    const real* K[6];
    real coef[6];
    int nk;
};

template <typename real>
__global__ void k_adj_lincomb(real* __restrict__ out, const real* __restrict__ s, LinComb<real> lc, long long len) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < len; q += (long long)gridDim.x * blockDim.x) {
        real acc = s[q];
        for (int l = 0; l < lc.nk; ++l)
            if (lc.coef[l] != real(0)) acc += lc.coef[l] * lc.K[l][q];
        out[q] = acc;
    }
}

// Pulse and renormalisation transposes, then lam_K_j = b_j lam_y and lam_s = lam_y.
template <typename real>
struct TopArgs {
    real* lam;           // in: dL/ds_after; out: lam_s = lam_y
    const real* y;       // unnormalised RK result
    real* LK[6];
    real b[6];
    int S;
    int renorm, pulse;
    uint64_t seed, replica;
    long long k;
    real sigma;
};

template <typename real>
__global__ void k_adj_top(TopArgs<real> a, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        real l0 = a.lam[i], l1 = a.lam[N + i], l2 = a.lam[2 * N + i];
        if (a.pulse) {
            const Words4 w = noise_words(a.seed, (uint64_t)i, (uint64_t)a.k, a.replica);
            real g0, g1, g2;
            Gauss<real>::draw(w, g0, g1, g2);
            pulse_rotate<real>(l0, l1, l2, -a.sigma * g0, -a.sigma * g1, -a.sigma * g2);
        }
        if (a.renorm) {
            const real y0 = a.y[i], y1 = a.y[N + i], y2 = a.y[2 * N + i];
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
        for (int j = 0; j < a.S; ++j) {
            a.LK[j][i] = a.b[j] * l0;
            a.LK[j][N + i] = a.b[j] * l1;
            a.LK[j][2 * N + i] = a.b[j] * l2;
        }
    }
}

// Stage transpose, site-local part: w and u at every site for v = dt lam_K,
// plus FP64 block partials of <w, sum_nn x> (J), 2 x_z w_z (D) and w (H) and
// the per-site field gradient gh += w.
template <typename real, bool PREC, bool HSITE>
__global__ void __launch_bounds__(kAT) k_adj_w(const real* __restrict__ x, const real* __restrict__ hs,
                                               const real* __restrict__ LK, real* __restrict__ w, real* __restrict__ u,
                                               double* __restrict__ gh, double* __restrict__ partials, int nx, int ny,
                                               int nz, real J, real twoD, real H0, real H1, real H2, real lambda,
                                               real dt, int bc) {
    __shared__ double red[kAT / 32];
    const long long N = (long long)nx * ny * nz;
    const real H[3] = {H0, H1, H2};
    double pJ = 0, pD = 0, pH0 = 0, pH1 = 0, pH2 = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        long long nb[6];
        neighbours(i, nx, ny, nz, nb);
        real wn[6];
        neighbour_weights<real>(i, nx, ny, nz, bc, wn);
        real hr[3];
        heff_at<real, HSITE>(x, hs, i, nb, wn, N, J, twoD, H, hr);
        // the transpose in the state precision (like the forward stages);
        // the parameter gradients accumulate in FP64
        const real s[3] = {x[i], x[N + i], x[2 * N + i]};
        const real v[3] = {dt * LK[i], dt * LK[N + i], dt * LK[2 * N + i]};
        real a[3], sv[3], ssv[3], hv[3], av[3], hsv[3];
        cross3r(s, hr, a);
        cross3r(s, v, sv);
        cross3r(s, sv, ssv);
        cross3r(hr, v, hv);
        cross3r(a, v, av);
        cross3r(hr, sv, hsv);
        real wi[3], ui[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (PREC) {
                wi[c] = -sv[c] - lambda * ssv[c];
                ui[c] = hv[c] - lambda * av[c] + lambda * hsv[c];
            } else {
                wi[c] = -lambda * ssv[c];
                ui[c] = -lambda * av[c] + lambda * hsv[c];
            }
            w[c * N + i] = wi[c];
            u[c * N + i] = ui[c];
            if (gh) gh[c * N + i] += (double)wi[c];
        }
        real sn[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const real* q = x + c * N;
            sn[c] = wn[0] * q[nb[0]] + wn[1] * q[nb[1]] + wn[2] * q[nb[2]] + wn[3] * q[nb[3]] + wn[4] * q[nb[4]] +
                    wn[5] * q[nb[5]];
        }
        pJ += (double)(wi[0] * sn[0] + wi[1] * sn[1] + wi[2] * sn[2]);
        pD += (double)(real(2) * s[2] * wi[2]);
        pH0 += (double)wi[0];
        pH1 += (double)wi[1];
        pH2 += (double)wi[2];
    }
    // each block adds into its own FP64 record, launch after launch in stream
    // order (deterministic); the records are summed once after the backward pass
    const double vals[5] = {pJ, pD, pH0, pH1, pH2};
    for (int q = 0; q < 5; ++q) {
        const double t = block_sum<double>(vals[q], red);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * 5 + q] += t;
    }
}

// Stage transpose, neighbour part: lx = u + J sum_nn w + 2D w_z z, then
// lam_s += lx and lam_K_l += a_jl lx for l < j.
template <typename real>
struct XArgs {
    const real* w;
    const real* u;
    real* lam;
    real* LK[6];
    real a[6];
    int nl;
    real J, twoD;
    int bc;
};

template <typename real>
__global__ void k_adj_x(XArgs<real> a, int nx, int ny, int nz) {
    const long long N = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        long long nb[6];
        neighbours(i, nx, ny, nz, nb);
        real wn[6];
        neighbour_weights<real>(i, nx, ny, nz, a.bc, wn);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const real* q = a.w + c * N;
            real lx = a.u[c * N + i] + a.J * (wn[0] * q[nb[0]] + wn[1] * q[nb[1]] + wn[2] * q[nb[2]] + wn[3] * q[nb[3]] +
                                              wn[4] * q[nb[4]] + wn[5] * q[nb[5]]);
            if (c == 2) lx += a.twoD * a.w[2 * N + i];
            a.lam[c * N + i] += lx;
            for (int l = 0; l < a.nl; ++l)
                if (a.a[l] != real(0)) a.LK[l][c * N + i] += a.a[l] * lx;
        }
    }
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
        neighbours(i, nx, ny, nz, nb);
        real wn[6];
        neighbour_weights<real>(i, nx, ny, nz, bc, wn);
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

size_t adjoint_workspace_bytes(const Geom& g, int elt, int stages, int K) {
    const size_t comp = (size_t)3 * (size_t)g.N() * (size_t)elt;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    size_t b = 0;
    b += al(comp) * (size_t)(K + 1);     // segment states
    b += al(comp) * (size_t)stages * 3;  // X_j, K_j, lam_K_j
    b += al(comp) * 5;                   // y, lam, w, u, scratch
    b += al(sizeof(double) * 5 * (size_t)adjoint_blocks(g));
    b += al(sizeof(double) * 8);         // accumulators
    b += al(sizeof(long long));          // pulse-number slot
    return b;
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
    real* w = reinterpret_cast<real*>(ws + off);
    off += al(compb);
    real* u = reinterpret_cast<real*>(ws + off);
    off += al(compb);
    off += al(compb);  // scratch
    const int nb = adjoint_blocks(g);
    double* partials = reinterpret_cast<double*>(ws + off);
    off += al(sizeof(double) * 5 * (size_t)nb);
    double* acc = reinterpret_cast<double*>(ws + off);
    off += al(sizeof(double) * 8);
    long long* kslot = reinterpret_cast<long long*>(ws + off);
    cudaStream_t st = A.stream;
    const real J = (real)A.J, twoD = (real)(2.0 * A.D), H0 = (real)A.H[0], H1 = (real)A.H[1], H2 = (real)A.H[2];
    const real lamb = (real)A.lambda, dt = (real)A.dt;
    const real* hs = A.h_site;
    const bool HS = hs != nullptr;
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
        // restore checkpoint and recompute the segment with the forward kernels
        e = cudaMemcpyAsync(seg, A.store + (size_t)sgi * len, compb, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        for (int m = 1; m <= seglen; ++m) {
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
            e = launch_step<real>(L);
            if (e != cudaSuccess) return e;
        }
        // transposed steps, last to first
        for (int m = seglen; m >= 1; --m) {
            const long long n = start + m;
            const bool pul = A.noise && (n % A.R) == (A.R / 2);
            const real* s = seg + (size_t)(m - 1) * len;
            // stages X_j and K_j = dt f(X_j), and y = s + sum b_j K_j
            for (int j = 0; j < S; ++j) {
                LinComb<real> lc{};
                for (int l = 0; l < j; ++l) {
                    lc.K[l] = Kst[l];
                    lc.coef[l] = (real)tb.a[j][l];
                }
                lc.nk = j;
                k_adj_lincomb<real><<<grid_for(len), kAT, 0, st>>>(X[j], s, lc, len);
                if (A.precession) {
                    if (HS) k_adj_rhs<real, true, true><<<grid_for(N), kAT, 0, st>>>(X[j], hs, Kst[j], g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                    else k_adj_rhs<real, true, false><<<grid_for(N), kAT, 0, st>>>(X[j], nullptr, Kst[j], g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                } else {
                    if (HS) k_adj_rhs<real, false, true><<<grid_for(N), kAT, 0, st>>>(X[j], hs, Kst[j], g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                    else k_adj_rhs<real, false, false><<<grid_for(N), kAT, 0, st>>>(X[j], nullptr, Kst[j], g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                }
            }
            {
                LinComb<real> lc{};
                for (int l = 0; l < S; ++l) {
                    lc.K[l] = Kst[l];
                    lc.coef[l] = (real)tb.b[l];
                }
                lc.nk = S;
                k_adj_lincomb<real><<<grid_for(len), kAT, 0, st>>>(y, s, lc, len);
            }
            TopArgs<real> ta{};
            ta.lam = lam;
            ta.y = y;
            for (int j = 0; j < S; ++j) {
                ta.LK[j] = LK[j];
                ta.b[j] = (real)tb.b[j];
            }
            ta.S = S;
            ta.renorm = A.renorm;
            ta.pulse = pul ? 1 : 0;
            ta.seed = A.seed;
            ta.replica = A.replica;
            ta.k = (n - 1) / A.R;
            ta.sigma = (real)A.sigma;
            k_adj_top<real><<<grid_for(N), kAT, 0, st>>>(ta, N);
            for (int j = S - 1; j >= 0; --j) {
                if (A.precession) {
                    if (HS) k_adj_w<real, true, true><<<nb, kAT, 0, st>>>(X[j], hs, LK[j], w, u, A.g_h, partials, g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                    else k_adj_w<real, true, false><<<nb, kAT, 0, st>>>(X[j], nullptr, LK[j], w, u, A.g_h, partials, g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                } else {
                    if (HS) k_adj_w<real, false, true><<<nb, kAT, 0, st>>>(X[j], hs, LK[j], w, u, A.g_h, partials, g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                    else k_adj_w<real, false, false><<<nb, kAT, 0, st>>>(X[j], nullptr, LK[j], w, u, A.g_h, partials, g.nx, g.ny, g.nz, J, twoD, H0, H1, H2, lamb, dt, A.bc);
                }
                XArgs<real> xa{};
                xa.w = w;
                xa.u = u;
                xa.lam = lam;
                for (int l = 0; l < j; ++l) {
                    xa.LK[l] = LK[l];
                    xa.a[l] = (real)tb.a[j][l];
                }
                xa.nl = j;
                xa.J = J;
                xa.twoD = twoD;
                xa.bc = A.bc;
                k_adj_x<real><<<grid_for(N), kAT, 0, st>>>(xa, g.nx, g.ny, g.nz);
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
