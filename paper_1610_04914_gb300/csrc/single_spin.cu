// Single-spin replicas (paper Sec. III: a spin in a field, and a uniaxial spin
// in a transverse field with its thermally activated escape, Sec. III.B).
// One thread owns one replica and integrates it through many steps in
// registers, with the pulse noise of Eqs. (phi_n) and (s_rotation) once per
// noise interval, or with the rectangular noise of Eq. (zeta_n) -- a random
// field in the precession term held over each interval, the conventional
// scheme the paper compares with (Sec. III.A).  Two kernels:
//   k_single_run     a fixed stretch of steps on the global step count n,
//                    optionally stopping at the first step after which
//                    s_z < 0 (the paper's first-passage procedure) and
//                    optionally summing s_z at the end of every interval
//                    (equilibrium averages, Fig. 4);
//   k_single_escape  renewal form of the first-passage procedure: a replica
//                    that crosses s_z = 0 records the passage time and
//                    restarts from the initial state as a new trial at the
//                    next interval start, so that no lane of a warp idles
//                    for long while the slowest trial of the warp runs on.
// The energy is E = -D s_z^2 - H.s, so H_eff = H + 2 D s_z z.  Noise counter
// of pulse k: (0, k, r, 0) for replica r in the run kernel (a one-site
// lattice with replica index r); (0, k, r + j nrep, 0) for trial j of replica
// r in the escape kernel, k counted from the trial's start.  Both kernels
// follow the pulse schedule of the global step count, so that the pulse
// branch is the same for all lanes of a warp.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/spinpulse.h"
#include "spin_device.cuh"
#include "spin_internal.h"

namespace spin {
namespace {

template <typename real>
struct SingleCommon {
    real* sx;
    real* sy;
    real* sz;
    const real* sigma;   // per replica: sqrt(2 lambda_r T_r Delta t), or sqrt(2 lambda_r T_r / Delta t) (RECT)
    const real* lambda;  // per replica damping
    int nrep, R, renorm, noise;
    real D2, Hx, Hy, Hz, dt;
    real a[6][6];
    real b[6];
    uint64_t seed;
};

// Which stage couplings a_jl and weights b_j of each integrator are nonzero
// (RK4, Butcher RK5, RK2 midpoint, Heun: the structure of the tableaus of
// tableau_for, whose values the kernels read); zero terms are skipped at
// compile time.  tableau_mask_matches checks the two agree before a launch.
__host__ __device__ constexpr int integ_stages(int integ) { return integ == 0 ? 4 : integ == 1 ? 6 : 2; }
__host__ __device__ constexpr bool a_nonzero(int integ, int j, int l) {
    return integ == 0 ? l == j - 1
         : integ == 1 ? !((j == 3 && l == 0) || (j == 4 && (l == 1 || l == 2)))
                      : (j == 1 && l == 0);
}
__host__ __device__ constexpr bool b_nonzero(int integ, int j) {
    return integ == 1 ? j != 1 : integ == 2 ? j == 1 : true;
}

bool tableau_mask_matches(int integ, const Tableau& tb) {
    if (tb.stages != integ_stages(integ)) return false;
    for (int j = 0; j < tb.stages; ++j) {
        if (!b_nonzero(integ, j) && tb.b[j] != 0.0) return false;
        for (int l = 0; l < j; ++l)
            if (!a_nonzero(integ, j, l) && tb.a[j][l] != 0.0) return false;
    }
    return true;
}

// One step of integrator INTEG on one spin, then |s| = 1.  RECT:
// the rectangular-noise field z is added to H_eff in the precession term of
// every stage (Eqs. (LLL), (zeta_n)); otherwise the noiseless equation.
template <typename real, bool PREC, int INTEG, bool RECT>
__device__ __forceinline__ void single_step(real& s0, real& s1, real& s2, real lam, const SingleCommon<real>& C,
                                            real z0, real z1, real z2) {
    constexpr int ST = integ_stages(INTEG);
    real K[ST][3];
#pragma unroll
    for (int j = 0; j < ST; ++j) {
        real x0 = s0, x1 = s1, x2 = s2;
#pragma unroll
        for (int l = 0; l < j; ++l) {
            if (!a_nonzero(INTEG, j, l)) continue;
            const real c = C.a[j][l];
            x0 += c * K[l][0];
            x1 += c * K[l][1];
            x2 += c * K[l][2];
        }
        real f0, f1, f2;
        if (RECT)
            llg_rhs_noise<real>(x0, x1, x2, C.Hx, C.Hy, C.Hz + C.D2 * x2, z0, z1, z2, lam, f0, f1, f2);
        else
            llg_rhs<real, PREC>(x0, x1, x2, C.Hx, C.Hy, C.Hz + C.D2 * x2, lam, f0, f1, f2);
        K[j][0] = C.dt * f0;
        K[j][1] = C.dt * f1;
        K[j][2] = C.dt * f2;
    }
#pragma unroll
    for (int j = 0; j < ST; ++j) {
        if (!b_nonzero(INTEG, j)) continue;
        s0 += C.b[j] * K[j][0];
        s1 += C.b[j] * K[j][1];
        s2 += C.b[j] * K[j][2];
    }
    if (C.renorm) {
        const real inv = Math<real>::rsqrt_(s0 * s0 + s1 * s1 + s2 * s2);
        s0 *= inv;
        s1 *= inv;
        s2 *= inv;
    }
}

// Rectangular-noise field of interval k: zeta = zs G(seed, 0, k, replica).
template <typename real>
__device__ __forceinline__ void draw_zeta(const SingleCommon<real>& C, uint64_t k, uint64_t replica, real zs,
                                          real& z0, real& z1, real& z2) {
    Gauss<real>::draw(noise_words(C.seed, 0ULL, k, replica), z0, z1, z2);
    z0 *= zs;
    z1 *= zs;
    z2 *= zs;
}

template <typename real>
struct RunArgs {
    SingleCommon<real> c;
    long long* first_passage;  // nullable; -1 = no passage yet
    double* sz_sum;            // nullable
    long long* sz_count;       // nullable with sz_sum
    long long n0, nsteps;
    int stop;
};

template <typename real, bool PREC, int INTEG, bool RECT>
__global__ void __launch_bounds__(128) k_single_run(RunArgs<real> A) {
    const SingleCommon<real>& C = A.c;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= C.nrep) return;
    long long fp = A.first_passage ? A.first_passage[r] : -1;
    if (A.stop && fp >= 0) return;
    real s0 = C.sx[r], s1 = C.sy[r], s2 = C.sz[r];
    const real sig = C.sigma[r], lam = C.lambda[r];
    double acc = 0.0;
    long long cnt = 0;
    // position in the schedule, advanced without a division per step:
    // ph = n mod R and kq = n div R for the step n just completed
    int ph = (int)(A.n0 % C.R);
    long long kq = A.n0 / C.R;
    const int half = C.R / 2;
    real z0 = 0, z1 = 0, z2 = 0;
    if (RECT && ph != 0) draw_zeta<real>(C, (uint64_t)kq, (uint64_t)r, sig, z0, z1, z2);  // mid-interval start
    for (long long n = A.n0 + 1; n <= A.n0 + A.nsteps; ++n) {
        if (RECT && ph == 0) draw_zeta<real>(C, (uint64_t)kq, (uint64_t)r, sig, z0, z1, z2);  // interval (n-1) div R
        single_step<real, PREC, INTEG, RECT>(s0, s1, s2, lam, C, z0, z1, z2);
        if (++ph == C.R) {
            ph = 0;
            ++kq;
        }
        // pulse number (n - 1) div R: kq, or kq - 1 when n is a multiple of R
        if (!RECT && C.noise && ph == half)
            pulse_site<real>(s0, s1, s2, C.seed, 0ULL, (uint64_t)(ph == 0 ? kq - 1 : kq), (uint64_t)r, sig);
        if (A.sz_sum && ph == 0) {
            acc += (double)s2;
            ++cnt;
        }
        if (A.stop && s2 < real(0)) {
            fp = n;
            break;
        }
    }
    C.sx[r] = s0;
    C.sy[r] = s1;
    C.sz[r] = s2;
    if (A.first_passage) A.first_passage[r] = fp;
    if (A.sz_sum) {
        A.sz_sum[r] += acc;
        A.sz_count[r] += cnt;
    }
}

template <typename real>
struct EscapeArgs {
    SingleCommon<real> c;
    long long* trial;       // per replica: index j of the running (or next) trial
    long long* local_step;  // per replica: steps done in the running trial; -1 = waiting
    long long* fpt_sum;     // per replica: sum of the passage steps of finished trials
    double* fpt_sq;         // nullable: sum of their squares
    long long* fpt_count;   // per replica: number of finished trials
    real i0, i1, i2;        // initial state of every trial
    long long n0, nsteps;   // global steps completed before this launch; steps to run
};

// The pulse schedule runs on the global step count n, the same for every
// lane of a warp, so the pulse branch never diverges; a replica that crossed
// waits (computing on its stale state, which is discarded) until the next
// n with n mod R == 0 and starts its next trial there, so that every trial
// sees the schedule of a fresh run: pulse after local step R/2 of each
// interval, pulse number counted from the trial's start.
template <typename real, bool PREC, int INTEG, bool RECT>
__global__ void __launch_bounds__(128) k_single_escape(EscapeArgs<real> A) {
    const SingleCommon<real>& C = A.c;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= C.nrep) return;
    real s0 = C.sx[r], s1 = C.sy[r], s2 = C.sz[r];
    const real sig = C.sigma[r], lam = C.lambda[r];
    long long j = A.trial[r], m = A.local_step[r];
    long long fsum = 0, fcnt = 0;
    double fsq = 0.0;
    int ph = (int)(A.n0 % C.R);  // global phase n mod R, advanced without a division per step
    const int half = C.R / 2;
    // a running trial must be in phase with the global schedule; one that is
    // not (inconsistent caller state) waits for the next interval start
    bool running = m >= 0 && (int)(m % C.R) == ph;
    if (!running) m = -1;
    long long mk = running ? m / C.R : 0;  // completed intervals of the running trial
    const uint64_t rep0 = (uint64_t)r;
    const uint64_t nrep = (uint64_t)C.nrep;
    real z0 = 0, z1 = 0, z2 = 0;
    if (RECT && ph != 0) draw_zeta<real>(C, (uint64_t)mk, rep0 + (uint64_t)j * nrep, sig, z0, z1, z2);
    for (long long it = 0; it < A.nsteps; ++it) {
        if (RECT && ph == 0) draw_zeta<real>(C, (uint64_t)mk, rep0 + (uint64_t)j * nrep, sig, z0, z1, z2);
        single_step<real, PREC, INTEG, RECT>(s0, s1, s2, lam, C, z0, z1, z2);
        if (++ph == C.R) ph = 0;
        m += running;
        mk += running && ph == 0;
        if (!RECT && C.noise && ph == half)
            pulse_site<real>(s0, s1, s2, C.seed, 0ULL, (uint64_t)(ph == 0 ? mk - 1 : mk), rep0 + (uint64_t)j * nrep,
                             sig);
        if (running && s2 < real(0)) {
            fsum += m;
            fsq += (double)m * (double)m;
            ++fcnt;
            ++j;
            running = false;
            m = -1;
        }
        if (!running && ph == 0) {
            running = true;
            m = 0;
            mk = 0;
            s0 = A.i0;
            s1 = A.i1;
            s2 = A.i2;
        }
    }
    C.sx[r] = s0;
    C.sy[r] = s1;
    C.sz[r] = s2;
    A.trial[r] = j;
    A.local_step[r] = m;
    A.fpt_sum[r] += fsum;
    A.fpt_count[r] += fcnt;
    if (A.fpt_sq) A.fpt_sq[r] += fsq;
}

template <typename real>
SingleCommon<real> make_common(const spin_params* p, int nrep, void* s, void* scratch) {
    SingleCommon<real> C{};
    real* base = static_cast<real*>(s);
    C.sx = base;
    C.sy = base + nrep;
    C.sz = base + 2 * (size_t)nrep;
    C.sigma = static_cast<const real*>(scratch);
    C.lambda = static_cast<const real*>(scratch) + nrep;
    C.nrep = nrep;
    C.R = p->steps_per_pulse;
    C.renorm = p->renorm;
    C.noise = p->noise;
    const Tableau tb = tableau_for(p->integrator);
    for (int j = 0; j < 6; ++j) {
        C.b[j] = (real)tb.b[j];
        for (int l = 0; l < 6; ++l) C.a[j][l] = (real)tb.a[j][l];
    }
    C.D2 = (real)(2.0 * p->D);
    C.Hx = (real)p->H[0];
    C.Hy = (real)p->H[1];
    C.Hz = (real)p->H[2];
    C.dt = (real)p->dt;
    C.seed = p->seed;
    return C;
}

template <typename real, bool PREC, int INTEG, bool RECT>
struct RunK {
    static void launch(int blocks, cudaStream_t st, const RunArgs<real>& A) {
        k_single_run<real, PREC, INTEG, RECT><<<blocks, 128, 0, st>>>(A);
    }
};
template <typename real, bool PREC, int INTEG, bool RECT>
struct EscK {
    static void launch(int blocks, cudaStream_t st, const EscapeArgs<real>& A) {
        k_single_escape<real, PREC, INTEG, RECT><<<blocks, 128, 0, st>>>(A);
    }
};

// Launch Kern<real, PREC, integrator, RECT> for the integrator, the precession
// flag and the noise kind (rectangular noise needs the precession term).
template <typename real, template <typename, bool, int, bool> class Kern, typename Args>
cudaError_t dispatch(const spin_params* p, int nrep, const Args& A, cudaStream_t st) {
    const int blocks = (nrep + 127) / 128;
    if (!tableau_mask_matches(p->integrator, tableau_for(p->integrator))) return cudaErrorInvalidValue;
    const int ns = p->integrator;
    const bool prec = p->precession != 0;
    const bool rect = p->noise == 2;
#define SPIN_SINGLE_CASE(NS)                                     \
    case NS:                                                     \
        if (rect)                                                \
            Kern<real, true, NS, true>::launch(blocks, st, A);   \
        else if (prec)                                           \
            Kern<real, true, NS, false>::launch(blocks, st, A);  \
        else                                                     \
            Kern<real, false, NS, false>::launch(blocks, st, A); \
        break;
    switch (ns) {
        SPIN_SINGLE_CASE(0)
        SPIN_SINGLE_CASE(1)
        SPIN_SINGLE_CASE(2)
        SPIN_SINGLE_CASE(3)
        default:
            return cudaErrorInvalidValue;
    }
#undef SPIN_SINGLE_CASE
    return cudaGetLastError();
}

int check_single(const spin_params* p, int nrep, const void* s, const void* scratch) {
    if (!p || nrep < 1 || !s || !scratch) return SPIN_EINVAL;
    if (p->precision != 32 && p->precision != 64) return SPIN_EINVAL;
    if (p->steps_per_pulse < 1 || !std::isfinite(p->dt) || p->dt == 0.0) return SPIN_EINVAL;
    if (p->integrator < 0 || p->integrator > 3) return SPIN_EINVAL;
    if (p->noise < 0 || p->noise > 2 || (p->noise == 2 && !p->precession)) return SPIN_EINVAL;
    if (!std::isfinite(p->D) || !std::isfinite(p->H[0]) || !std::isfinite(p->H[1]) || !std::isfinite(p->H[2]))
        return SPIN_EINVAL;
    return SPIN_OK;
}

// Upload the per-replica noise scales (computed in FP64) and dampings into
// the caller's scratch: the pulse angle scale sqrt(2 lambda_r T_r Delta t),
// Eq. (phi_n), or the rectangular field scale sqrt(2 lambda_r T_r / Delta t),
// Eq. (zeta_n).
template <typename real>
cudaError_t upload_scales(const spin_params* p, int nrep, const double* T, const double* lambda, void* scratch,
                          cudaStream_t st) {
    const double Dt = p->steps_per_pulse * std::fabs(p->dt);
    std::vector<real> h(2 * (size_t)nrep);
    for (int r = 0; r < nrep; ++r) {
        const double lam = lambda ? lambda[r] : p->lambda;
        h[r] = (real)(p->noise == 2 ? std::sqrt(2.0 * lam * T[r] / Dt) : std::sqrt(2.0 * lam * T[r] * Dt));
        h[nrep + r] = (real)lam;
    }
    cudaError_t e = cudaMemcpyAsync(scratch, h.data(), sizeof(real) * h.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

template <typename real>
cudaError_t run_t(const spin_params* p, int nrep, void* s, void* scratch, long long n0, long long nsteps, int stop,
                  long long* fp, double* sz_sum, long long* sz_count, cudaStream_t st) {
    RunArgs<real> A{};
    A.c = make_common<real>(p, nrep, s, scratch);
    A.first_passage = fp;
    A.sz_sum = sz_sum;
    A.sz_count = sz_count;
    A.n0 = n0;
    A.nsteps = nsteps;
    A.stop = stop;
    return dispatch<real, RunK>(p, nrep, A, st);
}

template <typename real>
cudaError_t escape_t(const spin_params* p, int nrep, const double* s_init, void* s, void* scratch, long long n0,
                     long long nsteps, long long* trial, long long* local_step, long long* fpt_sum, double* fpt_sq,
                     long long* fpt_count, cudaStream_t st) {
    EscapeArgs<real> A{};
    A.c = make_common<real>(p, nrep, s, scratch);
    A.trial = trial;
    A.local_step = local_step;
    A.fpt_sum = fpt_sum;
    A.fpt_sq = fpt_sq;
    A.fpt_count = fpt_count;
    A.i0 = (real)s_init[0];
    A.i1 = (real)s_init[1];
    A.i2 = (real)s_init[2];
    A.n0 = n0;
    A.nsteps = nsteps;
    return dispatch<real, EscK>(p, nrep, A, st);
}

}  // namespace
}  // namespace spin

extern "C" int spin_single_prepare(const spin_params* p, int32_t nrep, const double* T, const double* lambda,
                                   void* scratch, void* cuda_stream) {
    using namespace spin;
    if (!p || nrep < 1 || !T || !scratch) return SPIN_EINVAL;
    if (p->precision != 32 && p->precision != 64) return SPIN_EINVAL;
    if (p->steps_per_pulse < 1 || !std::isfinite(p->dt) || p->dt == 0.0) return SPIN_EINVAL;
    if (p->noise < 0 || p->noise > 2) return SPIN_EINVAL;
    for (int r = 0; r < nrep; ++r) {
        const double lam = lambda ? lambda[r] : p->lambda;
        if (!(T[r] >= 0.0) || !std::isfinite(T[r]) || !(lam >= 0.0) || !std::isfinite(lam)) return SPIN_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const cudaError_t e = p->precision == 64 ? upload_scales<double>(p, nrep, T, lambda, scratch, st)
                                             : upload_scales<float>(p, nrep, T, lambda, scratch, st);
    return e == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

extern "C" int spin_single_run(const spin_params* p, int32_t nrep, void* s, void* scratch, int64_t n0,
                               int64_t nsteps, int32_t stop_on_crossing, int64_t* first_passage, double* sz_sum,
                               int64_t* sz_count, void* cuda_stream) {
    using namespace spin;
    const int chk = check_single(p, nrep, s, scratch);
    if (chk != SPIN_OK) return chk;
    if (n0 < 0 || nsteps < 0 || (sz_sum == nullptr) != (sz_count == nullptr)) return SPIN_EINVAL;
    if (stop_on_crossing && !first_passage) return SPIN_EINVAL;
    if (nsteps == 0) return SPIN_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const cudaError_t e =
        p->precision == 64
            ? run_t<double>(p, nrep, s, scratch, n0, nsteps, stop_on_crossing, (long long*)first_passage, sz_sum,
                            (long long*)sz_count, st)
            : run_t<float>(p, nrep, s, scratch, n0, nsteps, stop_on_crossing, (long long*)first_passage, sz_sum,
                           (long long*)sz_count, st);
    return e == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

extern "C" int spin_single_escape(const spin_params* p, int32_t nrep, const double* s_init, void* s, void* scratch,
                                  int64_t n0, int64_t nsteps, int64_t* trial, int64_t* local_step, int64_t* fpt_sum,
                                  double* fpt_sq, int64_t* fpt_count, void* cuda_stream) {
    using namespace spin;
    const int chk = check_single(p, nrep, s, scratch);
    if (chk != SPIN_OK) return chk;
    if (!s_init || n0 < 0 || nsteps < 0 || !trial || !local_step || !fpt_sum || !fpt_count) return SPIN_EINVAL;
    if (!std::isfinite(s_init[0]) || !std::isfinite(s_init[1]) || !std::isfinite(s_init[2]) || !(s_init[2] >= 0.0))
        return SPIN_EINVAL;
    if (nsteps == 0) return SPIN_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const cudaError_t e =
        p->precision == 64
            ? escape_t<double>(p, nrep, s_init, s, scratch, n0, nsteps, (long long*)trial, (long long*)local_step,
                               (long long*)fpt_sum, fpt_sq, (long long*)fpt_count, st)
            : escape_t<float>(p, nrep, s_init, s, scratch, n0, nsteps, (long long*)trial, (long long*)local_step,
                              (long long*)fpt_sum, fpt_sq, (long long*)fpt_count, st);
    return e == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}
