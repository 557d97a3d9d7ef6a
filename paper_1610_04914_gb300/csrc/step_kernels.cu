// One integration step delta t of the noiseless Landau-Lifshitz equation,
// Eq. (LLL), on the periodic simple-cubic lattice, followed by
// renormalisation and, on pulse steps, the noise rotation of Eq. (s_rotation).
//
// Two paths:
//  * chain tableaus (RK4, RK2 midpoint, Heun: stage j needs only K_{j-1}):
//    one fused kernel per step.  Each CTA owns an (x, y) tile plus a halo of
//    S sites (S = number of stages) and marches along z.  At wavefront
//    iteration t it loads spin plane t+S from HBM, evaluates stage j on plane
//    t+S-j for j = 1..S (x-y neighbours of each stage input through shared
//    memory, z neighbours from per-thread register rings) and writes the
//    finished plane t.  Stage states never leave the SM: one read and one
//    write of the state per step.
//  * Butcher RK5 in FP32 without a per-site field: two fused three-stage
//    segments (step_rk5.cu).
//  * any tableau, any precision: one stencil kernel per stage plus a combine
//    kernel, stage states in the workspace.
#include <cuda_runtime.h>

#include <algorithm>

#include "spin_device.cuh"
#include "spin_internal.h"

namespace spin {

__host__ __device__ inline int wrap_index(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

Tableau tableau_for(int integrator) {
    Tableau t{};
    switch (integrator) {
        case 0:  // classical RK4
            t.stages = 4;
            t.a[1][0] = 0.5;
            t.a[2][1] = 0.5;
            t.a[3][2] = 1.0;
            t.b[0] = 1.0 / 6.0;
            t.b[1] = 2.0 / 6.0;
            t.b[2] = 2.0 / 6.0;
            t.b[3] = 1.0 / 6.0;
            t.chain = true;
            break;
        case 1:  // Butcher's RK5 as listed in the paper's Appendix
            t.stages = 6;
            t.a[1][0] = 0.25;
            t.a[2][0] = 0.125;
            t.a[2][1] = 0.125;
            t.a[3][1] = -0.5;
            t.a[3][2] = 1.0;
            t.a[4][0] = 3.0 / 16.0;
            t.a[4][3] = 9.0 / 16.0;
            t.a[5][0] = -3.0 / 7.0;
            t.a[5][1] = 2.0 / 7.0;
            t.a[5][2] = 12.0 / 7.0;
            t.a[5][3] = -12.0 / 7.0;
            t.a[5][4] = 8.0 / 7.0;
            t.b[0] = 7.0 / 90.0;
            t.b[2] = 32.0 / 90.0;
            t.b[3] = 12.0 / 90.0;
            t.b[4] = 32.0 / 90.0;
            t.b[5] = 7.0 / 90.0;
            t.chain = false;
            break;
        case 2:  // RK2 midpoint
            t.stages = 2;
            t.a[1][0] = 0.5;
            t.b[1] = 1.0;
            t.chain = true;
            break;
        default:  // Heun
            t.stages = 2;
            t.a[1][0] = 1.0;
            t.b[0] = 0.5;
            t.b[1] = 0.5;
            t.chain = true;
            break;
    }
    return t;
}

// ---------------------------------------------------------------------------
// Fused chain-tableau step
// ---------------------------------------------------------------------------

template <typename real>
struct ChainArgs {
    const real* __restrict__ in0;
    const real* __restrict__ in1;
    const real* __restrict__ in2;
    real* __restrict__ out0;
    real* __restrict__ out1;
    real* __restrict__ out2;
    const real* __restrict__ hs0;
    const real* __restrict__ hs1;
    const real* __restrict__ hs2;
    int nx, ny, nz, tz, n_iter;
    real J, twoD, Hx, Hy, Hz, lambda;
    real cdt[4];  // x_{j+1} = s + cdt[j-1] f_j   (dt folded in)
    real bdt[4];  // s' = s + sum_j bdt[j-1] f_j
    int renorm;
    uint64_t seed, replica;
    real sigma;
    const long long* interval;
    int bc;  // 1: free boundaries (outside columns and planes are zero spins)
};

// Register rings, indexed by (local plane index) & 3.
template <typename real, int S, bool HSITE>
struct Rings {
    real s[4][3];
    real x[S > 1 ? S - 1 : 1][4][3];  // x_j for j = 2..S
    real y[4][3];
    real h[HSITE ? 4 : 1][3];
};

template <typename real, int S, int BX, int BY, bool PREC, bool HSITE, bool PULSE, int P>
__device__ __forceinline__ void chain_iteration(const ChainArgs<real>& a, Rings<real, S, HSITE>& r,
                                                real* __restrict__ sh, int i, int t0, int z0, int col,
                                                int plane, bool out_col, int tx, int ty, int xm, int xp,
                                                int ym, int yp, long long k, real cmask) {
    constexpr int TILE = BX * BY;
    const int buf = P & 1;
    real* shb = sh + buf * (S * 3 * TILE);
    const int me = ty * BX + tx;

    // 1. publish this iteration's stage inputs for the x-y neighbours
#pragma unroll
    for (int j = 1; j <= S; ++j) {
        const int slot = (P + S - j) & 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const real v = (j == 1) ? r.s[slot][c] : r.x[j - 2][slot][c];
            shb[((j - 1) * 3 + c) * TILE + me] = v;
        }
    }

    // 2. stream in spin plane t+S (and the site field one plane behind)
    const int t = i + t0;
    {
        const int gz = wrap_index(t + S, a.nz);
        const long long off = (long long)gz * plane + col;
        const int slot = (P + S) & 3;
        r.s[slot][0] = __ldg(a.in0 + off);
        r.s[slot][1] = __ldg(a.in1 + off);
        r.s[slot][2] = __ldg(a.in2 + off);
        if (a.bc) {
            const real m = (t + S >= 0 && t + S < a.nz) ? cmask : real(0);
            r.s[slot][0] *= m;
            r.s[slot][1] *= m;
            r.s[slot][2] *= m;
        }
        if (HSITE) {
            const int gzh = wrap_index(t + S - 1, a.nz);
            const long long offh = (long long)gzh * plane + col;
            const int sl = (P + S - 1) & 3;
            r.h[sl][0] = __ldg(a.hs0 + offh);
            r.h[sl][1] = __ldg(a.hs1 + offh);
            r.h[sl][2] = __ldg(a.hs2 + offh);
        }
    }
    __syncthreads();

    // 3. stage j on plane t+S-j, j = 1..S
#pragma unroll
    for (int j = 1; j <= S; ++j) {
        const int slot = (P + S - j) & 3;
        const int sm = (slot + 3) & 3, sp = (slot + 1) & 3;
        const real* shj = shb + (j - 1) * 3 * TILE;
        real cen[3], sum[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const real* q = shj + c * TILE;
            cen[c] = (j == 1) ? r.s[slot][c] : r.x[j - 2][slot][c];
            const real zmv = (j == 1) ? r.s[sm][c] : r.x[j - 2][sm][c];
            const real zpv = (j == 1) ? r.s[sp][c] : r.x[j - 2][sp][c];
            // neighbour order x-1, x+1, y-1, y+1, z-1, z+1
            sum[c] = q[ty * BX + xm] + q[ty * BX + xp] + q[ym * BX + tx] + q[yp * BX + tx] + zmv + zpv;
        }
        real hx = a.J * sum[0] + a.Hx;
        real hy = a.J * sum[1] + a.Hy;
        real hz = a.J * sum[2] + a.Hz;
        if (HSITE) {
            hx += r.h[slot][0];
            hy += r.h[slot][1];
            hz += r.h[slot][2];
        }
        hz += a.twoD * cen[2];
        real f[3];
        llg_rhs<real, PREC>(cen[0], cen[1], cen[2], hx, hy, hz, a.lambda, f[0], f[1], f[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (j == 1)
                r.y[slot][c] = r.s[slot][c] + a.bdt[0] * f[c];
            else
                r.y[slot][c] = r.y[slot][c] + a.bdt[j - 1] * f[c];
            if (j < S) r.x[j - 1][slot][c] = r.s[slot][c] + a.cdt[j - 1] * f[c];
        }
        if (j == S) {
            // finished plane t
            if (out_col && t >= z0 && t < z0 + a.tz && t < a.nz) {
                real ox = r.y[slot][0], oy = r.y[slot][1], oz = r.y[slot][2];
                if (a.renorm) {
                    const real inv = Math<real>::rsqrt_(ox * ox + oy * oy + oz * oz);
                    ox *= inv;
                    oy *= inv;
                    oz *= inv;
                }
                const long long site = (long long)t * plane + col;
                if (PULSE) pulse_site<real>(ox, oy, oz, a.seed, (uint64_t)site, (uint64_t)k, a.replica, a.sigma);
                a.out0[site] = ox;
                a.out1[site] = oy;
                a.out2[site] = oz;
            }
        }
    }
}

template <typename real, int S, int BX, int BY, bool PREC, bool HSITE, bool PULSE>
__global__ void __launch_bounds__(BX* BY, 1) k_step_chain(ChainArgs<real> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* sh = reinterpret_cast<real*>(smem_raw);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gxu = (int)blockIdx.x * (BX - 2 * S) - S + tx;
    const int gyu = (int)blockIdx.y * (BY - 2 * S) - S + ty;
    const int gx = wrap_index(gxu, a.nx), gy = wrap_index(gyu, a.ny);
    const bool out_col = tx >= S && tx < BX - S && ty >= S && ty < BY - S && gxu < a.nx && gyu < a.ny;
    const int col = gy * a.nx + gx;
    const int plane = a.nx * a.ny;
    const int xm = tx > 0 ? tx - 1 : tx, xp = tx < BX - 1 ? tx + 1 : tx;
    const int ym = ty > 0 ? ty - 1 : ty, yp = ty < BY - 1 ? ty + 1 : ty;
    const int z0 = (int)blockIdx.z * a.tz;
    const int t0 = z0 - 2 * S + 2;
    const long long k = PULSE ? *a.interval : 0;
    const real cmask = (a.bc && (gxu < 0 || gxu >= a.nx || gyu < 0 || gyu >= a.ny)) ? real(0) : real(1);

    Rings<real, S, HSITE> r;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            r.s[q][c] = real(0);
            r.y[q][c] = real(0);
#pragma unroll
            for (int j = 0; j < (S > 1 ? S - 1 : 1); ++j) r.x[j][q][c] = real(0);
            if (HSITE) r.h[q][c] = real(0);
        }
    // preload s at local planes S-2 and S-1
#pragma unroll
    for (int L = S - 2; L <= S - 1; ++L) {
        const long long off = (long long)wrap_index(t0 + L, a.nz) * plane + col;
        r.s[L & 3][0] = __ldg(a.in0 + off);
        r.s[L & 3][1] = __ldg(a.in1 + off);
        r.s[L & 3][2] = __ldg(a.in2 + off);
        if (a.bc) {
            const real m = (t0 + L >= 0 && t0 + L < a.nz) ? cmask : real(0);
            r.s[L & 3][0] *= m;
            r.s[L & 3][1] *= m;
            r.s[L & 3][2] *= m;
        }
    }

    for (int i = 0; i < a.n_iter; i += 4) {
        chain_iteration<real, S, BX, BY, PREC, HSITE, PULSE, 0>(a, r, sh, i + 0, t0, z0, col, plane, out_col, tx, ty, xm, xp, ym, yp, k, cmask);
        chain_iteration<real, S, BX, BY, PREC, HSITE, PULSE, 1>(a, r, sh, i + 1, t0, z0, col, plane, out_col, tx, ty, xm, xp, ym, yp, k, cmask);
        chain_iteration<real, S, BX, BY, PREC, HSITE, PULSE, 2>(a, r, sh, i + 2, t0, z0, col, plane, out_col, tx, ty, xm, xp, ym, yp, k, cmask);
        chain_iteration<real, S, BX, BY, PREC, HSITE, PULSE, 3>(a, r, sh, i + 3, t0, z0, col, plane, out_col, tx, ty, xm, xp, ym, yp, k, cmask);
    }
}

template <typename real, int S, int BX, int BY, bool PREC, bool HSITE, bool PULSE>
static cudaError_t launch_chain_t(const ChainArgs<real>& a, dim3 grid, cudaStream_t st) {
    const size_t smem = sizeof(real) * 2 * S * 3 * BX * BY;
    k_step_chain<real, S, BX, BY, PREC, HSITE, PULSE><<<grid, dim3(BX, BY), smem, st>>>(a);
    return cudaGetLastError();
}

template <typename real, int S, int BX, int BY, bool PREC, bool HSITE, bool PULSE>
static cudaError_t prepare_chain_t() {
    const size_t smem = sizeof(real) * 2 * S * 3 * BX * BY;
    return cudaFuncSetAttribute(k_step_chain<real, S, BX, BY, PREC, HSITE, PULSE>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename real, int S, int BX, int BY>
static cudaError_t dispatch_chain(const ChainArgs<real>& a, dim3 grid, cudaStream_t st, bool prec, bool hsite,
                                  bool pulse, bool prepare) {
#define SPIN_CHAIN_CASE(P_, H_, U_)                                                     \
    if (prepare) {                                                                      \
        cudaError_t e = prepare_chain_t<real, S, BX, BY, P_, H_, U_>();                 \
        if (e != cudaSuccess) return e;                                                 \
    } else if (prec == P_ && hsite == H_ && pulse == U_) {                              \
        return launch_chain_t<real, S, BX, BY, P_, H_, U_>(a, grid, st);                \
    }
    SPIN_CHAIN_CASE(true, false, false)
    SPIN_CHAIN_CASE(true, false, true)
    SPIN_CHAIN_CASE(true, true, false)
    SPIN_CHAIN_CASE(true, true, true)
    SPIN_CHAIN_CASE(false, false, false)
    SPIN_CHAIN_CASE(false, false, true)
    SPIN_CHAIN_CASE(false, true, false)
    SPIN_CHAIN_CASE(false, true, true)
#undef SPIN_CHAIN_CASE
    return prepare ? cudaSuccess : cudaErrorInvalidValue;
}

// CTA shape of the fused step: 32x16 columns for float, 16x16 for double
// (the double register rings need up to 255 registers per thread).
template <typename real>
struct ChainShape;
template <>
struct ChainShape<float> {
    static constexpr int BX = 32, BY = 16;
};
template <>
struct ChainShape<double> {
    static constexpr int BX = 16, BY = 16;
};

template <typename real>
cudaError_t prepare_step_kernels() {
    constexpr int BX = ChainShape<real>::BX, BY = ChainShape<real>::BY;
    ChainArgs<real> a{};
    cudaError_t e = dispatch_chain<real, 4, BX, BY>(a, dim3(1), 0, false, false, false, true);
    if (e != cudaSuccess) return e;
    e = dispatch_chain<real, 2, BX, BY>(a, dim3(1), 0, false, false, false, true);
    if (e != cudaSuccess || sizeof(real) != 4) return e;
    if ((e = prepare_patch_kernels()) != cudaSuccess) return e;
    return prepare_rk5_kernels();
}
template cudaError_t prepare_step_kernels<float>();
template cudaError_t prepare_step_kernels<double>();

template <typename real>
static cudaError_t launch_chain(const StepLaunch<real>& L) {
    constexpr int BX = ChainShape<real>::BX, BY = ChainShape<real>::BY;
    const Tableau& tb = *L.tab;
    const int S = tb.stages;
    ChainArgs<real> a{};
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
        a.cdt[j] = (j + 1 < S) ? (real)(tb.a[j + 1][j] * L.dt) : real(0);
        a.bdt[j] = (j < S) ? (real)(tb.b[j] * L.dt) : real(0);
    }
    a.renorm = L.renorm;
    a.seed = L.seed;
    a.replica = L.replica;
    a.sigma = L.sigma;
    a.interval = L.d_interval;
    a.bc = L.bc;
    const int tiles_x = (L.g.nx + (BX - 2 * S) - 1) / (BX - 2 * S);
    const int tiles_y = (L.g.ny + (BY - 2 * S) - 1) / (BY - 2 * S);
    // z chunk: enough CTAs to fill the GPU twice over, chunks of >= 8 planes
    int zc = L.g.nz;
    const int want = 2 * 152;
    while (zc > 8 && (long long)tiles_x * tiles_y * ((L.g.nz + zc - 1) / zc) < want) zc = (zc + 1) / 2;
    a.tz = zc;
    const int iters = zc + 2 * S - 2;
    a.n_iter = (iters + 3) & ~3;
    dim3 grid(tiles_x, tiles_y, (L.g.nz + zc - 1) / zc);
    const bool hs = L.hs[0] != nullptr;
    const bool prec = L.precession != 0;
    if (S == 4) return dispatch_chain<real, 4, BX, BY>(a, grid, L.stream, prec, hs, L.pulse != 0, false);
    if (S == 2) return dispatch_chain<real, 2, BX, BY>(a, grid, L.stream, prec, hs, L.pulse != 0, false);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Generic tableau: stencil-per-stage kernels
// ---------------------------------------------------------------------------

template <typename real>
struct Vec3P {
    const real* p[3];
};

// K = dt f(x) over the lattice; neighbours read from global memory.  Blocks
// of kGX threads along x on a (x tile, row) grid: one integer division per row
// (y, z), none per site; periodic neighbours wrap by comparison.
constexpr int kGX = 128;

template <typename real, bool PREC, bool HSITE>
__global__ void __launch_bounds__(kGX) k_stage_rhs(Vec3P<real> x, Vec3P<real> hs, real* __restrict__ K0,
                                                   real* __restrict__ K1, real* __restrict__ K2, int nx, int ny,
                                                   int nz, Phys<real> ph, real dt, int bc) {
    const int xi = blockIdx.x * kGX + threadIdx.x;
    if (xi >= nx) return;
    const long long P = (long long)nx * ny;
    const long long N = P * nz;
    const int rows = ny * nz;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int zi = row / ny;
        const int yi = row - zi * ny;
        const long long i = (long long)row * nx + xi;
        const long long nb[6] = {xi > 0 ? i - 1 : i + (nx - 1),
                                 xi < nx - 1 ? i + 1 : i - (nx - 1),
                                 yi > 0 ? i - nx : i + (long long)(ny - 1) * nx,
                                 yi < ny - 1 ? i + nx : i - (long long)(ny - 1) * nx,
                                 zi > 0 ? i - P : i + (N - P),
                                 zi < nz - 1 ? i + P : i - (N - P)};
        // free boundaries: a neighbour across a face does not exist
        const real w[6] = {(bc && xi == 0) ? real(0) : real(1), (bc && xi == nx - 1) ? real(0) : real(1),
                           (bc && yi == 0) ? real(0) : real(1), (bc && yi == ny - 1) ? real(0) : real(1),
                           (bc && zi == 0) ? real(0) : real(1), (bc && zi == nz - 1) ? real(0) : real(1)};
        real h[3], s[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const real* q = x.p[c];
            const real sum = w[0] * q[nb[0]] + w[1] * q[nb[1]] + w[2] * q[nb[2]] + w[3] * q[nb[3]] + w[4] * q[nb[4]] +
                             w[5] * q[nb[5]];
            h[c] = ph.J * sum + ph.H[c];
            if (HSITE) h[c] += hs.p[c][i];
            s[c] = q[i];
        }
        h[2] += ph.twoD * s[2];
        real f[3];
        llg_rhs<real, PREC>(s[0], s[1], s[2], h[0], h[1], h[2], ph.lambda, f[0], f[1], f[2]);
        K0[i] = dt * f[0];
        K1[i] = dt * f[1];
        K2[i] = dt * f[2];
    }
}

template <typename real>
struct CombineArgs {
    const real* s[3];
    const real* K[6];  // each K[l] points at 3N: components at K[l] + c*N
    real coef[6];
    int nk;
    real* out[3];
    int renorm, pulse;
    uint64_t seed, replica;
    real sigma;
    const long long* interval;
};

// out = s + sum_l coef[l] K_l, optionally renormalised and pulsed.  The term
// count NK is a template argument (dispatched on the host), so the pointer
// table is indexed with constants and stays in the kernel parameters.
template <typename real, int NK>
__global__ void k_combine(CombineArgs<real> a, long long N) {
    const long long k = a.pulse ? *a.interval : 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        real v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            real acc = a.s[c][i];
#pragma unroll
            for (int l = 0; l < NK; ++l)
                if (a.coef[l] != real(0)) acc += a.coef[l] * a.K[l][c * N + i];
            v[c] = acc;
        }
        if (a.renorm) {
            const real inv = Math<real>::rsqrt_(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            v[0] *= inv;
            v[1] *= inv;
            v[2] *= inv;
        }
        if (a.pulse) pulse_site<real>(v[0], v[1], v[2], a.seed, (uint64_t)i, (uint64_t)k, a.replica, a.sigma);
        a.out[0][i] = v[0];
        a.out[1][i] = v[1];
        a.out[2][i] = v[2];
    }
}

template <typename real>
static void launch_combine(int nk, const CombineArgs<real>& c, long long N, int blocks, int threads, cudaStream_t st) {
    switch (nk) {
        case 1: k_combine<real, 1><<<blocks, threads, 0, st>>>(c, N); break;
        case 2: k_combine<real, 2><<<blocks, threads, 0, st>>>(c, N); break;
        case 3: k_combine<real, 3><<<blocks, threads, 0, st>>>(c, N); break;
        case 4: k_combine<real, 4><<<blocks, threads, 0, st>>>(c, N); break;
        case 5: k_combine<real, 5><<<blocks, threads, 0, st>>>(c, N); break;
        default: k_combine<real, 6><<<blocks, threads, 0, st>>>(c, N); break;
    }
}

template <typename real>
static cudaError_t launch_generic(const StepLaunch<real>& L) {
    const Tableau& tb = *L.tab;
    const long long N = L.g.N();
    const int threads = 256;
    const int blocks = (int)std::min<long long>((N + threads - 1) / threads, 152LL * 16);
    // tmp layout: K_1..K_S (3N each), then x (3N)
    real* K[6];
    for (int j = 0; j < tb.stages; ++j) K[j] = L.tmp + (size_t)j * 3 * N;
    real* xs = L.tmp + (size_t)tb.stages * 3 * N;
    const bool hs = L.hs[0] != nullptr;
    Vec3P<real> hv{{L.hs[0], L.hs[1], L.hs[2]}};
    const long long rows = (long long)L.g.ny * L.g.nz;
    const dim3 rgrid((L.g.nx + kGX - 1) / kGX, (unsigned)std::min<long long>(rows, 65535));
    for (int j = 0; j < tb.stages; ++j) {
        Vec3P<real> xv;
        if (j == 0) {
            xv = Vec3P<real>{{L.in[0], L.in[1], L.in[2]}};
        } else {
            CombineArgs<real> c{};
            for (int q = 0; q < 3; ++q) {
                c.s[q] = L.in[q];
                c.out[q] = xs + (size_t)q * N;
            }
            for (int l = 0; l < j; ++l) {
                c.K[l] = K[l];
                c.coef[l] = (real)tb.a[j][l];
            }
            c.nk = j;
            launch_combine<real>(j, c, N, blocks, threads, L.stream);
            xv = Vec3P<real>{{xs, xs + N, xs + 2 * N}};
        }
        real* k0 = K[j];
        if (L.precession) {
            if (hs)
                k_stage_rhs<real, true, true><<<rgrid, kGX, 0, L.stream>>>(xv, hv, k0, k0 + N, k0 + 2 * N, L.g.nx, L.g.ny, L.g.nz, L.ph, (real)L.dt, L.bc);
            else
                k_stage_rhs<real, true, false><<<rgrid, kGX, 0, L.stream>>>(xv, hv, k0, k0 + N, k0 + 2 * N, L.g.nx, L.g.ny, L.g.nz, L.ph, (real)L.dt, L.bc);
        } else {
            if (hs)
                k_stage_rhs<real, false, true><<<rgrid, kGX, 0, L.stream>>>(xv, hv, k0, k0 + N, k0 + 2 * N, L.g.nx, L.g.ny, L.g.nz, L.ph, (real)L.dt, L.bc);
            else
                k_stage_rhs<real, false, false><<<rgrid, kGX, 0, L.stream>>>(xv, hv, k0, k0 + N, k0 + 2 * N, L.g.nx, L.g.ny, L.g.nz, L.ph, (real)L.dt, L.bc);
        }
    }
    CombineArgs<real> c{};
    for (int q = 0; q < 3; ++q) {
        c.s[q] = L.in[q];
        c.out[q] = L.out[q];
    }
    for (int l = 0; l < tb.stages; ++l) {
        c.K[l] = K[l];
        c.coef[l] = (real)tb.b[l];
    }
    c.nk = tb.stages;
    c.renorm = L.renorm;
    c.pulse = L.pulse;
    c.seed = L.seed;
    c.replica = L.replica;
    c.sigma = L.sigma;
    c.interval = L.d_interval;
    launch_combine<real>(tb.stages, c, N, blocks, threads, L.stream);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_step(const StepLaunch<real>& L) {
    if (L.tab->chain && !L.force_generic && (L.tab->stages == 4 || L.tab->stages == 2)) {
        if (sizeof(real) == 4) return launch_step_patch(reinterpret_cast<const StepLaunch<float>&>(L));
        return launch_chain<real>(L);
    }
    if (sizeof(real) == 4 && !L.force_generic && rk5_fused_supports(reinterpret_cast<const StepLaunch<float>&>(L)))
        return launch_step_rk5(reinterpret_cast<const StepLaunch<float>&>(L));
    return launch_generic<real>(L);
}

template cudaError_t launch_step<float>(const StepLaunch<float>&);
template cudaError_t launch_step<double>(const StepLaunch<double>&);

// ---------------------------------------------------------------------------
// Noise draw on its own (verification entry point)
// ---------------------------------------------------------------------------

template <typename real>
__global__ void k_noise_draw(uint64_t seed, long long k, long long replica, long long n, uint64_t* words,
                             real* gauss) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const Words4 w = noise_words(seed, (uint64_t)i, (uint64_t)k, (uint64_t)replica);
        if (words) {
#pragma unroll
            for (int q = 0; q < 4; ++q) words[4 * i + q] = w.w[q];
        }
        if (gauss) {
            real g0, g1, g2;
            Gauss<real>::draw(w, g0, g1, g2);
            gauss[3 * i + 0] = g0;
            gauss[3 * i + 1] = g1;
            gauss[3 * i + 2] = g2;
        }
    }
}

cudaError_t launch_noise_draw(uint64_t seed, long long k, long long replica, long long n, int precision,
                              uint64_t* words, void* gauss, cudaStream_t stream) {
    const int threads = 256;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n + threads - 1) / threads, 152LL * 8));
    if (precision == 64)
        k_noise_draw<double><<<blocks, threads, 0, stream>>>(seed, k, replica, n, words, (double*)gauss);
    else
        k_noise_draw<float><<<blocks, threads, 0, stream>>>(seed, k, replica, n, words, (float*)gauss);
    return cudaGetLastError();
}

__global__ void k_set_counter(long long* d, long long v) { *d = v; }

cudaError_t launch_set_counter(long long* d, long long value, cudaStream_t stream) {
    k_set_counter<<<1, 1, 0, stream>>>(d, value);
    return cudaGetLastError();
}

}  // namespace spin
