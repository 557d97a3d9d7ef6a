// Checkerboard Metropolis Monte Carlo on the simple-cubic lattice (Sec. IV):
// the comparison method of the paper's many-spin experiment.  A trial moves
// s_i to (s_i + R u)/|s_i + R u| with u uniform on the sphere and is accepted
// if the energy change dE <= 0, else with probability exp(-dE/T).  The
// paper's sweep visits the sites one after another; here one sweep updates
// the sites with x+y+z even (colour 0) in one launch and then those with
// x+y+z odd (colour 1): no two sites of a colour are neighbours (periodic
// sizes even), so each launch updates its sites independently, one thread
// per site.  The random numbers of site i in sweep w are those of the
// sequential sweep: Philox4x64-10 with counter (i, w, replica, 0) and key
// (seed, "monte"); u from words 0 and 1 (cos(theta) = 2 u0 - 1,
// phi = 2 pi u1), the acceptance uniform from word 2.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/spinpulse.h"
#include "spin_device.cuh"
#include "spin_internal.h"

namespace spin {
namespace {

constexpr uint64_t kStreamMC = 0x6D6F6E7465ULL;  // "monte"

template <typename real>
struct MetroArgs {
    real* s0;
    real* s1;
    real* s2;
    const real* h0;  // per-site field, nullable
    const real* h1;
    const real* h2;
    int nx, ny, nz, bc, color;
    long long sweep;
    uint64_t seed, replica;
    real J, D, Hx, Hy, Hz, T, Rtrial;
    unsigned long long* accepted;  // nullable
};

__device__ __forceinline__ double uniform_d(uint64_t w) {
    return ((double)(w >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

template <typename real>
struct MetroMath;
// cos(theta) = 2 u0 - 1 and sin(theta) = sqrt(1 - cos(theta)^2) of the trial
// direction.  FP64 takes these literally.  FP32 forms the same reals from u0
// and 1 - u0 = ((~w >> 11) + 1/2) 2^-53, both rounded once from the 53-bit
// integer: cos = u0 - (1 - u0), sin = 2 sqrt(u0 (1 - u0)), so neither loses
// precision near the poles (rounding u0 itself near 1 would).
template <>
struct MetroMath<double> {
    __device__ __forceinline__ static double u(uint64_t w) { return uniform_d(w); }
    __device__ __forceinline__ static void polar(uint64_t w, double& c, double& s) {
        c = 2.0 * uniform_d(w) - 1.0;
        s = sqrt(1.0 - c * c);
    }
    __device__ __forceinline__ static void sincos2pi(double x, double* s, double* c) { sincospi(2.0 * x, s, c); }
    __device__ __forceinline__ static double exp_(double x) { return exp(x); }
    __device__ __forceinline__ static double sqrt_(double x) { return sqrt(x); }
};
template <>
struct MetroMath<float> {
    __device__ __forceinline__ static float u(uint64_t w) { return Gauss<float>::u01(w); }
    __device__ __forceinline__ static void polar(uint64_t w, float& c, float& s) {
        const float a = Gauss<float>::u01(w), b = Gauss<float>::u01(~w);  // u0 and 1 - u0
        c = a - b;
        s = 2.0f * sqrtf(a * b);
    }
    __device__ __forceinline__ static void sincos2pi(float x, float* s, float* c) { sincospif(2.0f * x, s, c); }
    __device__ __forceinline__ static float exp_(float x) { return expf(x); }
    __device__ __forceinline__ static float sqrt_(float x) { return sqrtf(x); }
};

template <typename real, bool HSITE>
__global__ void __launch_bounds__(256) k_metropolis(MetroArgs<real> A) {
    using M = MetroMath<real>;
    const int hx = (A.nx + 1) >> 1;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)A.ny * A.nz * hx;
    int acc = 0;
    if (t < total) {
        const int q = (int)(t % hx);
        const long long row = t / hx;
        const int y = (int)(row % A.ny);
        const int z = (int)(row / A.ny);
        const int x = 2 * q + ((y + z + A.color) & 1);
        if (x < A.nx) {
            const long long i = x + (long long)A.nx * (y + (long long)A.ny * z);
            const Words4 w = philox4x64_10((uint64_t)i, (uint64_t)A.sweep, A.replica, 0ULL, A.seed, kStreamMC);
            real cz, st, sp, cp;
            M::polar(w.w[0], cz, st);
            M::sincos2pi(M::u(w.w[1]), &sp, &cp);
            const real o0 = A.s0[i], o1 = A.s1[i], o2 = A.s2[i];
            real n0 = o0 + A.Rtrial * (st * cp), n1 = o1 + A.Rtrial * (st * sp), n2 = o2 + A.Rtrial * cz;
            const real nn = M::sqrt_(n0 * n0 + n1 * n1 + n2 * n2);
            n0 /= nn;
            n1 /= nn;
            n2 /= nn;
            // exchange field of the six neighbours (free boundaries: missing
            // neighbours contribute nothing)
            real l0 = 0, l1 = 0, l2 = 0;
            const long long sx = 1, sy = A.nx, sz = (long long)A.nx * A.ny;
            auto add = [&](long long j) {
                l0 += A.s0[j];
                l1 += A.s1[j];
                l2 += A.s2[j];
            };
            if (x > 0) add(i - sx); else if (!A.bc) add(i + (A.nx - 1) * sx);
            if (x < A.nx - 1) add(i + sx); else if (!A.bc) add(i - (A.nx - 1) * sx);
            if (y > 0) add(i - sy); else if (!A.bc) add(i + (A.ny - 1) * sy);
            if (y < A.ny - 1) add(i + sy); else if (!A.bc) add(i - (A.ny - 1) * sy);
            if (z > 0) add(i - sz); else if (!A.bc) add(i + (A.nz - 1) * sz);
            if (z < A.nz - 1) add(i + sz); else if (!A.bc) add(i - (A.nz - 1) * sz);
            l0 = A.J * l0 + A.Hx;
            l1 = A.J * l1 + A.Hy;
            l2 = A.J * l2 + A.Hz;
            if (HSITE) {
                l0 += A.h0[i];
                l1 += A.h1[i];
                l2 += A.h2[i];
            }
            const real e_old = -(o0 * l0 + o1 * l1 + o2 * l2) - A.D * o2 * o2;
            const real e_new = -(n0 * l0 + n1 * l1 + n2 * l2) - A.D * n2 * n2;
            const real dE = e_new - e_old;
            if (dE <= real(0) || M::u(w.w[2]) < M::exp_(-dE / A.T)) {
                A.s0[i] = n0;
                A.s1[i] = n1;
                A.s2[i] = n2;
                acc = 1;
            }
        }
    }
    if (A.accepted) {
        const unsigned cnt = __reduce_add_sync(0xffffffffu, (unsigned)acc);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(A.accepted, (unsigned long long)cnt);
    }
}

// Colour c of sweeps sweep0 .. sweep0+nsweeps-1 (c < 0: both colours, 0 then 1).
template <typename real>
cudaError_t sweeps_t(const spin_params* p, void* s, const void* h_site, uint64_t seed, double Rtrial,
                     long long sweep0, long long nsweeps, int only_color, unsigned long long* accepted,
                     cudaStream_t st) {
    MetroArgs<real> A{};
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    A.s0 = static_cast<real*>(s);
    A.s1 = A.s0 + N;
    A.s2 = A.s0 + 2 * N;
    if (h_site) {
        A.h0 = static_cast<const real*>(h_site);
        A.h1 = A.h0 + N;
        A.h2 = A.h0 + 2 * N;
    }
    A.nx = p->nx;
    A.ny = p->ny;
    A.nz = p->nz;
    A.bc = p->bc;
    A.seed = seed;
    A.replica = (uint64_t)p->replica;
    A.J = (real)p->J;
    A.D = (real)p->D;
    A.Hx = (real)p->H[0];
    A.Hy = (real)p->H[1];
    A.Hz = (real)p->H[2];
    A.T = (real)p->T;
    A.Rtrial = (real)Rtrial;
    A.accepted = accepted;
    const long long threads = (long long)p->ny * p->nz * ((p->nx + 1) / 2);
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    for (long long w = sweep0; w < sweep0 + nsweeps; ++w) {
        A.sweep = w;
        for (int c = 0; c < 2; ++c) {
            if (only_color >= 0 && c != only_color) continue;
            A.color = c;
            if (h_site)
                k_metropolis<real, true><<<blocks, 256, 0, st>>>(A);
            else
                k_metropolis<real, false><<<blocks, 256, 0, st>>>(A);
        }
    }
    return cudaGetLastError();
}

int check_metropolis(const spin_params* p, const void* s, double* R_trial) {
    if (!p || !s) return SPIN_EINVAL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return SPIN_EINVAL;
    if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return SPIN_EINVAL;
    if (p->precision != 32 && p->precision != 64) return SPIN_EINVAL;
    if (p->bc < 0 || p->bc > 1 || p->replica < 0) return SPIN_EINVAL;
    // periodic sizes must be even (two colours); a periodic size 1 would make a
    // site its own neighbour
    if (p->bc == 0 && ((p->nx & 1) || (p->ny & 1) || (p->nz & 1))) return SPIN_EINVAL;
    if (!(p->T > 0.0) || !std::isfinite(p->T) || !std::isfinite(p->J) || !std::isfinite(p->D)) return SPIN_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->H[a])) return SPIN_EINVAL;
    if (*R_trial <= 0.0) {
        if (!(p->J > 0.0)) return SPIN_EINVAL;
        *R_trial = 1.55 * std::sqrt(p->T / (6.0 * p->J));  // the paper's trial length, ~50% acceptance
    }
    if (!std::isfinite(*R_trial)) return SPIN_EINVAL;
    return SPIN_OK;
}

int metropolis(const spin_params* p, void* s, const void* h_site, uint64_t mc_seed, double R_trial,
               long long sweep0, long long nsweeps, int only_color, int64_t* accepted, void* cuda_stream) {
    const int chk = check_metropolis(p, s, &R_trial);
    if (chk != SPIN_OK) return chk;
    if (sweep0 < 0 || nsweeps < 0) return SPIN_EINVAL;
    if (nsweeps == 0) return SPIN_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(accepted);
    const cudaError_t e =
        p->precision == 64 ? sweeps_t<double>(p, s, h_site, mc_seed, R_trial, sweep0, nsweeps, only_color, acc, st)
                           : sweeps_t<float>(p, s, h_site, mc_seed, R_trial, sweep0, nsweeps, only_color, acc, st);
    return e == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

}  // namespace
}  // namespace spin

extern "C" int spin_metropolis_sweeps(const spin_params* p, void* s, const void* h_site, uint64_t mc_seed,
                                      double R_trial, int64_t sweep0, int64_t nsweeps, int64_t* accepted,
                                      void* cuda_stream) {
    return spin::metropolis(p, s, h_site, mc_seed, R_trial, sweep0, nsweeps, -1, accepted, cuda_stream);
}

extern "C" int spin_metropolis_color(const spin_params* p, void* s, const void* h_site, uint64_t mc_seed,
                                     double R_trial, int64_t sweep, int32_t color, int64_t* accepted,
                                     void* cuda_stream) {
    if (color != 0 && color != 1) return SPIN_EINVAL;
    return spin::metropolis(p, s, h_site, mc_seed, R_trial, sweep, 1, color, accepted, cuda_stream);
}
