/*
 * FP64 CPU oracle for the pulse-noise many-spin time step
 * (Garanin, "Pulse-noise approach for classical spin systems", arXiv:1610.04914).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, constant table or helper with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Everything is double precision, one site at a time, in the order the paper
 * states the algorithm.  Compile with -ffp-contract=off so that no fused
 * multiply-add changes the rounding of the written expressions.
 *
 * Units: gamma = mu0 = k_B = 1 (paper, end of Sec. II).
 *
 * Lattice: simple cubic nx*ny*nz, periodic or free boundaries (the paper's
 * particle of Sec. IV has free ones), site index i = x + nx*(y + ny*z).  Spin state is structure-of-arrays:
 * s[0*N+i] = s_x, s[1*N+i] = s_y, s[2*N+i] = s_z.
 *
 * Parity status of each function (what pins it) is listed beside it.
 *
 * The whole-lattice loops carry OpenMP pragmas over z-planes (or over array
 * elements): every site's value is computed by the same expression from the
 * same inputs whichever thread runs it, so a build with -fopenmp gives
 * bitwise the results of the serial build (checked by a test); without
 * -fopenmp the pragmas are ignored.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Parameters                                                                */
/* ------------------------------------------------------------------------ */

enum { ORC_RK4 = 0, ORC_RK5_BUTCHER = 1, ORC_RK2_MIDPOINT = 2, ORC_HEUN = 3 };

typedef struct {
    int32_t nx, ny, nz;
    int32_t integrator;      /* ORC_RK4 | ORC_RK5_BUTCHER | ORC_RK2_MIDPOINT | ORC_HEUN */
    int32_t precession;      /* 1: full LLL right-hand side; 0: slow (overdamped) equation */
    int32_t R;               /* steps per noise interval, R = Delta t / delta t >= 1 */
    int32_t renorm;          /* 1: s <- s/|s| after every full step */
    int32_t replica;         /* third Philox counter word */
    int32_t bc;              /* 0: periodic; 1: free (missing neighbours contribute nothing) */
    int32_t unused;
    double J, D, H[3];       /* exchange, uniaxial anisotropy (z), Zeeman field */
    double lambda, T, dt;    /* damping, temperature, integration step delta t */
    uint64_t seed;           /* Philox key word 0 for the noise pulses */
} orc_params;

/* Philox key word 1: one fixed value per random stream. */
#define ORC_STREAM_NOISE 0x6E6F697365ULL /* "noise" */
#define ORC_STREAM_MC    0x6D6F6E7465ULL /* "monte" */

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).                        */
/* Pinned against numpy.random.Philox (same generator), see tests.          */
/* ------------------------------------------------------------------------ */

static void mul_hilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    /* The two round multipliers and the two Weyl key increments of the
       4x64 variant, as published with the generator. */
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        mul_hilo64(M0, c0, &hi0, &lo0);
        mul_hilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Open-interval uniform from the top 53 bits: ((w >> 11) + 1/2) * 2^-53. */
static double u01(uint64_t w)
{
    return ((double)(w >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* Box-Muller (paper, Appendix): three unit normals from one Philox block.
   G0, G1 from (u0, u1); G2 from (u2, u3). */
void orc_gauss3(const uint64_t w[4], double G[3])
{
    const double two_pi = 6.283185307179586476925286766559;
    double u0 = u01(w[0]), u1 = u01(w[1]), u2 = u01(w[2]), u3 = u01(w[3]);
    double r0 = sqrt(-2.0 * log(u0));
    double r2 = sqrt(-2.0 * log(u2));
    G[0] = r0 * cos(two_pi * u1);
    G[1] = r0 * sin(two_pi * u1);
    G[2] = r2 * cos(two_pi * u3);
}

/* The Gaussian vector G_n of one site for pulse number k. */
void orc_noise_gauss(uint64_t seed, int64_t site, int64_t k, int64_t replica, double G[3])
{
    uint64_t ctr[4] = {(uint64_t)site, (uint64_t)k, (uint64_t)replica, 0};
    uint64_t key[2] = {seed, ORC_STREAM_NOISE};
    uint64_t w[4];
    orc_philox4x64(ctr, key, w);
    orc_gauss3(w, G);
}

/* ------------------------------------------------------------------------ */
/* Effective field (Eq. LLL's H_eff for the simple-cubic Heisenberg lattice) */
/*   H_eff,i = J sum_{j in nn(i)} s_j + 2 D s_{i,z} z + H + h_i              */
/* Pinned by: magnon dispersion, dE/dt = -lambda sum |s x H_eff|^2, the      */
/* uniform-state single-spin map, and the Metropolis equilibrium.           */
/* ------------------------------------------------------------------------ */

/* Index of site (x, y, z); with free boundaries a position outside the
   lattice has no site and gives -1. */
static int64_t site_index(const orc_params *p, int x, int y, int z)
{
    if (p->bc == 1 && (x < 0 || x >= p->nx || y < 0 || y >= p->ny || z < 0 || z >= p->nz)) return -1;
    x = (x % p->nx + p->nx) % p->nx;
    y = (y % p->ny + p->ny) % p->ny;
    z = (z % p->nz + p->nz) % p->nz;
    return (int64_t)x + (int64_t)p->nx * ((int64_t)y + (int64_t)p->ny * z);
}

static void heff_site(const orc_params *p, const double *s, const double *hsite,
                      int x, int y, int z, double Heff[3])
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    const int64_t nb[6] = {
        site_index(p, x - 1, y, z), site_index(p, x + 1, y, z),
        site_index(p, x, y - 1, z), site_index(p, x, y + 1, z),
        site_index(p, x, y, z - 1), site_index(p, x, y, z + 1),
    };
    const int64_t i = site_index(p, x, y, z);
    for (int a = 0; a < 3; ++a) {
        double sum = 0.0;
        for (int j = 0; j < 6; ++j)
            if (nb[j] >= 0) sum += s[a * N + nb[j]];
        Heff[a] = p->J * sum + p->H[a];
        if (hsite) Heff[a] += hsite[a * N + i];
    }
    Heff[2] += 2.0 * p->D * s[2 * N + i];
}

void orc_heff(const orc_params *p, const double *s, const double *hsite, double *Heff)
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                double h[3];
                int64_t i = site_index(p, x, y, z);
                heff_site(p, s, hsite, x, y, z, h);
                Heff[i] = h[0]; Heff[N + i] = h[1]; Heff[2 * N + i] = h[2];
            }
}

/* ------------------------------------------------------------------------ */
/* Right-hand side of the noiseless equation (Eq. LLL with zeta = 0):        */
/*   precessional: f = s x H_eff - lambda s x (s x H_eff)                    */
/*   slow (precession discarded, Sec. II): f = - lambda s x (s x H_eff)      */
/* ------------------------------------------------------------------------ */

static void cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Right-hand side of Eq. (LLL) at every site.  zeta (3N values or NULL) is
   the rectangular-noise field of Eq. (zeta_n); it enters the precession
   term only: f = s x (H_eff + zeta) - lambda s x (s x H_eff). */
static void rhs_field(const orc_params *p, const double *s, const double *hsite, const double *zeta, double *f)
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                int64_t i = site_index(p, x, y, z);
                double h[3], si[3] = {s[i], s[N + i], s[2 * N + i]};
                double sxh[3], sxsxh[3], hp[3], prec[3];
                heff_site(p, s, hsite, x, y, z, h);
                cross(si, h, sxh);
                cross(si, sxh, sxsxh);
                for (int a = 0; a < 3; ++a) hp[a] = h[a] + (zeta ? zeta[a * N + i] : 0.0);
                cross(si, hp, prec);
                for (int a = 0; a < 3; ++a) {
                    double damp = -p->lambda * sxsxh[a];
                    f[a * N + i] = p->precession ? (prec[a] + damp) : damp;
                }
            }
}

void orc_rhs(const orc_params *p, const double *s, const double *hsite, double *f)
{
    rhs_field(p, s, hsite, NULL, f);
}

/* ------------------------------------------------------------------------ */
/* One integration step delta t = h of the noiseless equation.               */
/* Tableaus: classical RK4 (textbook); Heun, RK2 midpoint and Butcher's RK5  */
/* as listed in the paper's Appendix.  Pinned by the convergence order and   */
/* the closed-form single-spin map.                                          */
/* ------------------------------------------------------------------------ */

/* y = x + sum_j c_j K_j over n arrays of length 3N */
static void lincomb(int64_t len, double *y, const double *x, int n,
                    const double *c, double *const *K)
{
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < len; ++q) {
        double acc = x[q];
        for (int j = 0; j < n; ++j) acc += c[j] * K[j][q];
        y[q] = acc;
    }
}

/* K = h * f(x); zeta is the rectangular-noise field (or NULL), the same in
   every stage of the step: the noise is held constant over its interval */
static void stage(const orc_params *p, const double *x, const double *hsite, const double *zeta, double *K)
{
    const int64_t len = 3LL * p->nx * p->ny * p->nz;
    rhs_field(p, x, hsite, zeta, K);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < len; ++q) K[q] *= p->dt;
}

void orc_renormalise(const orc_params *p, double *s)
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double n = sqrt(s[i] * s[i] + s[N + i] * s[N + i] + s[2 * N + i] * s[2 * N + i]);
        s[i] /= n; s[N + i] /= n; s[2 * N + i] /= n;
    }
}

static void integrate_field(const orc_params *p, double *s, const double *hsite, const double *zeta)
{
    const int64_t len = 3LL * p->nx * p->ny * p->nz;
    double *K[6], *xt = malloc(sizeof(double) * len);
    for (int j = 0; j < 6; ++j) K[j] = malloc(sizeof(double) * len);

    if (p->integrator == ORC_RK4) {
        /* K1 = h f(x); K2 = h f(x + K1/2); K3 = h f(x + K2/2); K4 = h f(x + K3);
           x <- x + (K1 + 2 K2 + 2 K3 + K4)/6 */
        double c2[1] = {0.5}, c3[1] = {0.5}, c4[1] = {1.0};
        stage(p, s, hsite, zeta, K[0]);
        lincomb(len, xt, s, 1, c2, &K[0]); stage(p, xt, hsite, zeta, K[1]);
        lincomb(len, xt, s, 1, c3, &K[1]); stage(p, xt, hsite, zeta, K[2]);
        lincomb(len, xt, s, 1, c4, &K[2]); stage(p, xt, hsite, zeta, K[3]);
        double b[4] = {1.0 / 6.0, 2.0 / 6.0, 2.0 / 6.0, 1.0 / 6.0};
        lincomb(len, s, s, 4, b, K);
    } else if (p->integrator == ORC_RK5_BUTCHER) {
        /* Butcher's RK5 (Appendix):
           K2 = h f(x + K1/4); K3 = h f(x + (K1+K2)/8); K4 = h f(x - K2/2 + K3);
           K5 = h f(x + 3(K1 + 3K4)/16);
           K6 = h f(x + (-3K1 + 2K2 + 12(K3-K4) + 8K5)/7);
           x <- x + (7K1 + 32K3 + 12K4 + 32K5 + 7K6)/90 */
        stage(p, s, hsite, zeta, K[0]);
        { double c[1] = {0.25}; lincomb(len, xt, s, 1, c, K); }
        stage(p, xt, hsite, zeta, K[1]);
        { double c[2] = {0.125, 0.125}; lincomb(len, xt, s, 2, c, K); }
        stage(p, xt, hsite, zeta, K[2]);
        { double c[3] = {0.0, -0.5, 1.0}; lincomb(len, xt, s, 3, c, K); }
        stage(p, xt, hsite, zeta, K[3]);
        { double c[4] = {3.0 / 16.0, 0.0, 0.0, 9.0 / 16.0}; lincomb(len, xt, s, 4, c, K); }
        stage(p, xt, hsite, zeta, K[4]);
        { double c[5] = {-3.0 / 7.0, 2.0 / 7.0, 12.0 / 7.0, -12.0 / 7.0, 8.0 / 7.0};
          lincomb(len, xt, s, 5, c, K); }
        stage(p, xt, hsite, zeta, K[5]);
        double b[6] = {7.0 / 90.0, 0.0, 32.0 / 90.0, 12.0 / 90.0, 32.0 / 90.0, 7.0 / 90.0};
        lincomb(len, s, s, 6, b, K);
    } else if (p->integrator == ORC_RK2_MIDPOINT) {
        /* K1 = h f(x); K2 = h f(x + K1/2); x <- x + K2 */
        double c[1] = {0.5};
        stage(p, s, hsite, zeta, K[0]);
        lincomb(len, xt, s, 1, c, K); stage(p, xt, hsite, zeta, K[1]);
        double b[2] = {0.0, 1.0};
        lincomb(len, s, s, 2, b, K);
    } else { /* ORC_HEUN: K1 = h f(x); K2 = h f(x + K1); x <- x + (K1 + K2)/2 */
        double c[1] = {1.0};
        stage(p, s, hsite, zeta, K[0]);
        lincomb(len, xt, s, 1, c, K); stage(p, xt, hsite, zeta, K[1]);
        double b[2] = {0.5, 0.5};
        lincomb(len, s, s, 2, b, K);
    }
    for (int j = 0; j < 6; ++j) free(K[j]);
    free(xt);
}

/* One step of the noiseless equation. */
void orc_integrate(const orc_params *p, double *s, const double *hsite)
{
    integrate_field(p, s, hsite, NULL);
}

/* ------------------------------------------------------------------------ */
/* Noise pulse: Eq. (phi_n) and the rotation formula Eq. (s_rotation).       */
/*   phi = sqrt(Lambda_N Delta t) G,  Lambda_N = 2 lambda T,  Delta t = R dt */
/*   s' = s cos(phi) + (n x s) sin(phi) + n (s.n)(1 - cos(phi))              */
/* Pinned by the exact one-pulse decay <s_z'> = s_z (1 + 2(1-sig^2)e^{-sig^2/2})/3 */
/* and by the Langevin-function equilibrium of independent spins.            */
/* ------------------------------------------------------------------------ */

double orc_pulse_sigma(const orc_params *p)
{
    double Lambda_N = 2.0 * p->lambda * p->T;
    double Delta_t = p->R * p->dt;
    return sqrt(Lambda_N * Delta_t);
}

void orc_rotate(const double phi_vec[3], double s[3])
{
    double phi = sqrt(phi_vec[0] * phi_vec[0] + phi_vec[1] * phi_vec[1] + phi_vec[2] * phi_vec[2]);
    if (phi == 0.0) return;
    double n[3] = {phi_vec[0] / phi, phi_vec[1] / phi, phi_vec[2] / phi};
    double nxs[3];
    cross(n, s, nxs);
    double sn = s[0] * n[0] + s[1] * n[1] + s[2] * n[2];
    double c = cos(phi), si = sin(phi);
    double out[3];
    for (int a = 0; a < 3; ++a) out[a] = s[a] * c + nxs[a] * si + n[a] * sn * (1.0 - c);
    s[0] = out[0]; s[1] = out[1]; s[2] = out[2];
}

/* Pulse number k (0-based) applied to every site. */
void orc_pulse(const orc_params *p, double *s, int64_t k)
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    const double sigma = orc_pulse_sigma(p);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double G[3], phi[3], si[3] = {s[i], s[N + i], s[2 * N + i]};
        orc_noise_gauss(p->seed, i, k, p->replica, G);
        for (int a = 0; a < 3; ++a) phi[a] = sigma * G[a];
        orc_rotate(phi, si);
        s[i] = si[0]; s[N + i] = si[1]; s[2 * N + i] = si[2];
    }
}

/* ------------------------------------------------------------------------ */
/* Observables, sampled at the end of each Delta t (Sec. III.A):             */
/*   M = (1/N) sum_i s_i                                                     */
/*   E = (1/N) [ -J sum_<ij> s_i.s_j - D sum_i s_iz^2 - sum_i (H + h_i).s_i ] */
/* with each nearest-neighbour bond counted once (3 forward bonds per site). */
/* Pinned by closed forms on uniform states and dE/dt = -lambda|s x H|^2.   */
/* ------------------------------------------------------------------------ */

void orc_observables(const orc_params *p, const double *s, const double *hsite, double out[4])
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    double M[3] = {0, 0, 0}, E = 0.0;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                int64_t i = site_index(p, x, y, z);
                int64_t fwd[3] = {site_index(p, x + 1, y, z), site_index(p, x, y + 1, z),
                                  site_index(p, x, y, z + 1)};
                double si[3] = {s[i], s[N + i], s[2 * N + i]};
                for (int a = 0; a < 3; ++a) M[a] += si[a];
                for (int b = 0; b < 3; ++b) {
                    int64_t j = fwd[b];
                    if (j < 0) continue;
                    E -= p->J * (si[0] * s[j] + si[1] * s[N + j] + si[2] * s[2 * N + j]);
                }
                E -= p->D * si[2] * si[2];
                for (int a = 0; a < 3; ++a) {
                    double field = p->H[a] + (hsite ? hsite[a * N + i] : 0.0);
                    E -= field * si[a];
                }
            }
    out[0] = M[0] / N; out[1] = M[1] / N; out[2] = M[2] / N; out[3] = E / N;
}

/* ------------------------------------------------------------------------ */
/* Pulse schedule (Eq. ST-expansion): steps are numbered n = 1, 2, ...; the   */
/* pulse follows step n when n mod R == floor(R/2) (for R = 1: every step),  */
/* its number is k = floor((n-1)/R); observables are sampled after steps     */
/* with n mod R == 0.                                                        */
/* ------------------------------------------------------------------------ */

int orc_is_pulse_step(int64_t n, int32_t R)
{
    return (n % R) == (R / 2);
}

int64_t orc_pulse_number(int64_t n, int32_t R)
{
    return (n - 1) / R;
}

/* Rectangular noise, Eq. (zeta_n): the field of interval k at every site,
   zeta_i = sqrt(2 lambda T / Delta t) G_i with the same Gaussian triple that
   pulse k would use (Delta t = R dt is the interval over which the field is
   held). */
void orc_rect_field(const orc_params *p, int64_t k, double *zeta)
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    const double scale = sqrt(2.0 * p->lambda * p->T / (p->R * fabs(p->dt)));
    for (int64_t i = 0; i < N; ++i) {
        double G[3];
        orc_noise_gauss(p->seed, i, k, p->replica, G);
        for (int a = 0; a < 3; ++a) zeta[a * N + i] = scale * G[a];
    }
}

/* Advance from step n0 (completed) by nsteps.  Writes one record
   (n, M_x, M_y, M_z, E) per sample into samples (capacity max_samples
   records) and returns the number written.  noise = 0: no noise;
   1: the pulses; 2: rectangular noise, the field of interval (n-1) div R in
   the precession term of step n (returns -1 when precession is off, since
   the noise has nowhere to enter). */
int64_t orc_run(const orc_params *p, double *s, const double *hsite,
                int64_t n0, int64_t nsteps, int noise,
                double *samples, int64_t max_samples)
{
    int64_t ns = 0;
    double *zeta = NULL;
    if (noise == 2) {
        if (!p->precession) return -1;
        zeta = malloc(sizeof(double) * 3 * (size_t)p->nx * p->ny * p->nz);
    }
    for (int64_t n = n0 + 1; n <= n0 + nsteps; ++n) {
        if (zeta && (n == n0 + 1 || (n - 1) % p->R == 0)) orc_rect_field(p, (n - 1) / p->R, zeta);
        integrate_field(p, s, hsite, zeta);
        if (p->renorm) orc_renormalise(p, s);
        if (noise == 1 && orc_is_pulse_step(n, p->R)) orc_pulse(p, s, orc_pulse_number(n, p->R));
        if (n % p->R == 0 && samples && ns < max_samples) {
            double o[4];
            orc_observables(p, s, hsite, o);
            samples[5 * ns + 0] = (double)n;
            samples[5 * ns + 1] = o[0];
            samples[5 * ns + 2] = o[1];
            samples[5 * ns + 3] = o[2];
            samples[5 * ns + 4] = o[3];
            ++ns;
        }
    }
    free(zeta);
    return ns;
}

/* ------------------------------------------------------------------------ */
/* Metropolis Monte Carlo (Sec. IV): sequential sweep in site order; trial   */
/* s' = (s + R u)/|s + R u| with u uniform on the sphere; accept if dE <= 0, */
/* else with probability exp(-dE/T).  The paper's trial length is           */
/* R = 1.55 sqrt(T/(6J)); the caller passes it (needed when J = 0).          */
/* Pinned by the Langevin function for independent spins.                    */
/* ------------------------------------------------------------------------ */

/* One Metropolis trial at site (x, y, z) in sweep sw; returns 1 if the
   trial was accepted (the spin then holds the trial direction). */
static int metro_site(const orc_params *p, double *s, const double *hsite, int x, int y, int z,
                      uint64_t mc_seed, double Rtrial, int64_t sw)
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    const double two_pi = 6.283185307179586476925286766559;
    int64_t i = site_index(p, x, y, z);
    uint64_t ctr[4] = {(uint64_t)i, (uint64_t)sw, (uint64_t)p->replica, 0};
    uint64_t key[2] = {mc_seed, ORC_STREAM_MC}, w[4];
    orc_philox4x64(ctr, key, w);
    double cz = 2.0 * u01(w[0]) - 1.0, ph = two_pi * u01(w[1]);
    double sz = sqrt(1.0 - cz * cz);
    double u[3] = {sz * cos(ph), sz * sin(ph), cz};
    double so[3] = {s[i], s[N + i], s[2 * N + i]}, sn[3];
    for (int a = 0; a < 3; ++a) sn[a] = so[a] + Rtrial * u[a];
    double nn = sqrt(sn[0] * sn[0] + sn[1] * sn[1] + sn[2] * sn[2]);
    for (int a = 0; a < 3; ++a) sn[a] /= nn;
    /* energy of site i with everything else fixed:
       -s_i.(J sum_nn s_j + H + h_i) - D s_iz^2 */
    double loc[3];
    const int64_t nb[6] = {
        site_index(p, x - 1, y, z), site_index(p, x + 1, y, z),
        site_index(p, x, y - 1, z), site_index(p, x, y + 1, z),
        site_index(p, x, y, z - 1), site_index(p, x, y, z + 1),
    };
    for (int a = 0; a < 3; ++a) {
        double sum = 0.0;
        for (int j = 0; j < 6; ++j) {
            /* a site that neighbours itself (lattice size 1)
               moves together with the trial spin */
            if (nb[j] == i || nb[j] < 0) continue;
            sum += s[a * N + nb[j]];
        }
        loc[a] = p->J * sum + p->H[a] + (hsite ? hsite[a * N + i] : 0.0);
    }
    double e_old = -(so[0] * loc[0] + so[1] * loc[1] + so[2] * loc[2]) - p->D * so[2] * so[2];
    double e_new = -(sn[0] * loc[0] + sn[1] * loc[1] + sn[2] * loc[2]) - p->D * sn[2] * sn[2];
    double dE = e_new - e_old;
    int accept = dE <= 0.0 || u01(w[2]) < exp(-dE / p->T);
    if (accept) {
        s[i] = sn[0]; s[N + i] = sn[1]; s[2 * N + i] = sn[2];
    }
    return accept;
}

static void record_series(const orc_params *p, const double *s, const double *hsite, double *row)
{
    double o[4];
    orc_observables(p, s, hsite, o);
    for (int a = 0; a < 4; ++a) row[a] = o[a];
}

int64_t orc_metropolis(const orc_params *p, double *s, const double *hsite,
                       uint64_t mc_seed, double Rtrial, int64_t sweep0, int64_t nsweeps,
                       double *series)
{
    int64_t accepted = 0;
    for (int64_t sw = sweep0; sw < sweep0 + nsweeps; ++sw) {
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x)
                    accepted += metro_site(p, s, hsite, x, y, z, mc_seed, Rtrial, sw);
        if (series) record_series(p, s, hsite, series + 4 * (sw - sweep0));
    }
    return accepted;
}

/* Checkerboard order: in sweep sw first every site with (x + y + z) even,
   then every site with (x + y + z) odd, each half in site order.  The two
   halves are independent sets (no two sites of one colour are neighbours)
   when every periodic dimension is even; the random numbers of a site are
   those of the sequential sweep, so only the order differs.
   orc_metropolis_color does one half (colour 0 or 1) of sweep sw. */
int64_t orc_metropolis_color(const orc_params *p, double *s, const double *hsite,
                             uint64_t mc_seed, double Rtrial, int64_t sw, int color)
{
    int64_t accepted = 0;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x)
                if (((x + y + z) & 1) == color)
                    accepted += metro_site(p, s, hsite, x, y, z, mc_seed, Rtrial, sw);
    return accepted;
}

int64_t orc_metropolis_checkerboard(const orc_params *p, double *s, const double *hsite,
                                    uint64_t mc_seed, double Rtrial, int64_t sweep0, int64_t nsweeps,
                                    double *series)
{
    int64_t accepted = 0;
    for (int64_t sw = sweep0; sw < sweep0 + nsweeps; ++sw) {
        accepted += orc_metropolis_color(p, s, hsite, mc_seed, Rtrial, sw, 0);
        accepted += orc_metropolis_color(p, s, hsite, mc_seed, Rtrial, sw, 1);
        if (series) record_series(p, s, hsite, series + 4 * (sw - sweep0));
    }
    return accepted;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint (pathwise, noise fixed) of the whole step: RK stages,    */
/* renormalisation and the pulse rotation, for losses of the final state     */
/* L = dLdE E(s_n) + dLdM . M(s_n).  Gradients w.r.t. J, D, H, h_i and s_0.  */
/* Pinned by central finite differences of L and by dot-product tests of    */
/* each primitive's transpose.                                               */
/* ------------------------------------------------------------------------ */

/* Butcher arrays of the integrators above: K_j = h f(x_j),
   x_j = x + sum_{l<j} a[j][l] K_l, x' = x + sum_j b[j] K_j. */
static int tableau(int integrator, double a[6][6], double b[6])
{
    memset(a, 0, sizeof(double) * 36);
    memset(b, 0, sizeof(double) * 6);
    if (integrator == ORC_RK4) {
        a[1][0] = 0.5; a[2][1] = 0.5; a[3][2] = 1.0;
        b[0] = 1.0 / 6.0; b[1] = 2.0 / 6.0; b[2] = 2.0 / 6.0; b[3] = 1.0 / 6.0;
        return 4;
    }
    if (integrator == ORC_RK5_BUTCHER) {
        a[1][0] = 0.25;
        a[2][0] = 0.125; a[2][1] = 0.125;
        a[3][1] = -0.5; a[3][2] = 1.0;
        a[4][0] = 3.0 / 16.0; a[4][3] = 9.0 / 16.0;
        a[5][0] = -3.0 / 7.0; a[5][1] = 2.0 / 7.0; a[5][2] = 12.0 / 7.0; a[5][3] = -12.0 / 7.0; a[5][4] = 8.0 / 7.0;
        b[0] = 7.0 / 90.0; b[2] = 32.0 / 90.0; b[3] = 12.0 / 90.0; b[4] = 32.0 / 90.0; b[5] = 7.0 / 90.0;
        return 6;
    }
    if (integrator == ORC_RK2_MIDPOINT) {
        a[1][0] = 0.5; b[1] = 1.0;
        return 2;
    }
    a[1][0] = 1.0; b[0] = 0.5; b[1] = 0.5; /* Heun */
    return 2;
}

/* out = J_f(x)^T v (f the right-hand side of Eq. LLL without noise), and
   the parameter gradients <v, df/dJ>, <v, df/dD>, <v, df/dH>, <v, df/dh_i>
   added into gJ, gD, gH, gh.  With w_i = (df_i/dH_i)^T v_i and
   u_i = (df_i/ds_i at fixed H)^T v_i:
     precessional: w = -(s x v) - lambda s x (s x v),
                   u = H x v - lambda a x v + lambda H x (s x v),  a = s x H
     slow:         w = -lambda s x (s x v),
                   u = -lambda a x v + lambda H x (s x v)
   and out_i = u_i + J sum_{j in nn(i)} w_j + 2D w_iz z. */
void orc_rhs_vjp(const orc_params *p, const double *x, const double *hsite, const double *v,
                 double *out, double *gJ, double *gD, double gH[3], double *gh)
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    double *w = malloc(sizeof(double) * 3 * N);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int xx = 0; xx < p->nx; ++xx) {
                int64_t i = site_index(p, xx, y, z);
                double H[3], si[3] = {x[i], x[N + i], x[2 * N + i]}, vi[3] = {v[i], v[N + i], v[2 * N + i]};
                heff_site(p, x, hsite, xx, y, z, H);
                double a[3], sv[3], ssv[3], wi[3], Hv[3], av[3], Hsv[3], ui[3];
                cross(si, H, a);
                cross(si, vi, sv);
                cross(si, sv, ssv);
                cross(H, vi, Hv);
                cross(a, vi, av);
                cross(H, sv, Hsv);
                for (int c = 0; c < 3; ++c) {
                    if (p->precession) {
                        wi[c] = -sv[c] - p->lambda * ssv[c];
                        ui[c] = Hv[c] - p->lambda * av[c] + p->lambda * Hsv[c];
                    } else {
                        wi[c] = -p->lambda * ssv[c];
                        ui[c] = -p->lambda * av[c] + p->lambda * Hsv[c];
                    }
                    w[c * N + i] = wi[c];
                    out[c * N + i] = ui[c];
                }
                /* parameter gradients */
                const int64_t nb[6] = {
                    site_index(p, xx - 1, y, z), site_index(p, xx + 1, y, z),
                    site_index(p, xx, y - 1, z), site_index(p, xx, y + 1, z),
                    site_index(p, xx, y, z - 1), site_index(p, xx, y, z + 1),
                };
                for (int c = 0; c < 3; ++c) {
                    double sum = 0.0;
                    for (int j = 0; j < 6; ++j)
                        if (nb[j] >= 0) sum += x[c * N + nb[j]];
                    if (gJ) *gJ += wi[c] * sum;
                    if (gH) gH[c] += wi[c];
                    if (gh) gh[c * N + i] += wi[c];
                }
                if (gD) *gD += 2.0 * si[2] * wi[2];
            }
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int xx = 0; xx < p->nx; ++xx) {
                int64_t i = site_index(p, xx, y, z);
                const int64_t nb[6] = {
                    site_index(p, xx - 1, y, z), site_index(p, xx + 1, y, z),
                    site_index(p, xx, y - 1, z), site_index(p, xx, y + 1, z),
                    site_index(p, xx, y, z - 1), site_index(p, xx, y, z + 1),
                };
                for (int c = 0; c < 3; ++c) {
                    double sum = 0.0;
                    for (int j = 0; j < 6; ++j)
                        if (nb[j] >= 0) sum += w[c * N + nb[j]];
                    out[c * N + i] += p->J * sum;
                }
                out[2 * N + i] += 2.0 * p->D * w[2 * N + i];
            }
    free(w);
}

/* Adjoint of one full step (integrate, renormalise, pulse k if pulse != 0)
   taken from state s: lam (3N) holds dL/ds_after on entry and dL/ds_before on
   exit; parameter gradients accumulate. */
void orc_step_vjp(const orc_params *p, const double *s, const double *hsite, int pulse, int64_t k,
                  double *lam, double *gJ, double *gD, double gH[3], double *gh)
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz, len = 3 * N;
    double A[6][6], B[6];
    const int S = tableau(p->integrator, A, B);
    double *X[6], *K[6], *LK[6];
    for (int j = 0; j < S; ++j) {
        X[j] = malloc(sizeof(double) * len);
        K[j] = malloc(sizeof(double) * len);
        LK[j] = calloc(len, sizeof(double));
    }
    double *yv = malloc(sizeof(double) * len), *lx = malloc(sizeof(double) * len);
    double *vv = malloc(sizeof(double) * len);
    /* forward recomputation of the stages */
    for (int j = 0; j < S; ++j) {
        for (int64_t q = 0; q < len; ++q) {
            double acc = s[q];
            for (int l = 0; l < j; ++l) acc += A[j][l] * K[l][q];
            X[j][q] = acc;
        }
        stage(p, X[j], hsite, NULL, K[j]);
    }
    for (int64_t q = 0; q < len; ++q) {
        double acc = s[q];
        for (int j = 0; j < S; ++j) acc += B[j] * K[j][q];
        yv[q] = acc;
    }
    /* pulse: lam <- R^T lam (rotation by -phi) */
    if (pulse) {
        const double sigma = orc_pulse_sigma(p);
        for (int64_t i = 0; i < N; ++i) {
            double G[3], phi[3], li[3] = {lam[i], lam[N + i], lam[2 * N + i]};
            orc_noise_gauss(p->seed, i, k, p->replica, G);
            for (int c = 0; c < 3; ++c) phi[c] = -sigma * G[c];
            orc_rotate(phi, li);
            lam[i] = li[0]; lam[N + i] = li[1]; lam[2 * N + i] = li[2];
        }
    }
    /* renormalisation: lam_y = (lam - u (u.lam)) / |y|, u = y/|y| */
    if (p->renorm) {
        for (int64_t i = 0; i < N; ++i) {
            double y3[3] = {yv[i], yv[N + i], yv[2 * N + i]};
            double n = sqrt(y3[0] * y3[0] + y3[1] * y3[1] + y3[2] * y3[2]);
            double u[3] = {y3[0] / n, y3[1] / n, y3[2] / n};
            double ul = u[0] * lam[i] + u[1] * lam[N + i] + u[2] * lam[2 * N + i];
            for (int c = 0; c < 3; ++c) lam[c * N + i] = (lam[c * N + i] - u[c] * ul) / n;
        }
    }
    /* RK stages in reverse: lam_s starts as lam_y, lam_K_j = b_j lam_y */
    for (int j = 0; j < S; ++j)
        for (int64_t q = 0; q < len; ++q) LK[j][q] = B[j] * lam[q];
    for (int j = S - 1; j >= 0; --j) {
        for (int64_t q = 0; q < len; ++q) vv[q] = p->dt * LK[j][q];  /* K_j = dt f(x_j) */
        orc_rhs_vjp(p, X[j], hsite, vv, lx, gJ, gD, gH, gh);
        for (int64_t q = 0; q < len; ++q) {
            lam[q] += lx[q];
            for (int l = 0; l < j; ++l) LK[l][q] += A[j][l] * lx[q];
        }
    }
    for (int j = 0; j < S; ++j) { free(X[j]); free(K[j]); free(LK[j]); }
    free(yv); free(lx); free(vv);
}

/* Gradients of L = dLdE E(s_n) + dLdM . M(s_n) after nsteps steps from s0
   (completed step count n0), all states kept in memory.  Writes
   *gJ, *gD, gH[3] (sums over the whole path including the explicit final-time
   terms), gh (3N, nullable) and gs0 (3N, nullable: dL/ds_0). */
void orc_adjoint(const orc_params *p, const double *s0, const double *hsite, int64_t n0, int64_t nsteps,
                 int noise, const double dLdM[3], double dLdE, double *gJ, double *gD, double gH[3],
                 double *gh, double *gs0)
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz, len = 3 * N;
    double *states = malloc(sizeof(double) * len * (nsteps + 1));
    memcpy(states, s0, sizeof(double) * len);
    for (int64_t m = 1; m <= nsteps; ++m) {
        double *cur = states + m * len;
        memcpy(cur, states + (m - 1) * len, sizeof(double) * len);
        int64_t n = n0 + m;
        orc_integrate(p, cur, hsite);
        if (p->renorm) orc_renormalise(p, cur);
        if (noise && orc_is_pulse_step(n, p->R)) orc_pulse(p, cur, orc_pulse_number(n, p->R));
    }
    const double *fin = states + nsteps * len;
    double *lam = malloc(sizeof(double) * len);
    double *Hf = malloc(sizeof(double) * len);
    orc_heff(p, fin, hsite, Hf);
    *gJ = 0.0; *gD = 0.0; gH[0] = gH[1] = gH[2] = 0.0;
    if (gh) memset(gh, 0, sizeof(double) * len);
    double bonds = 0.0, sz2 = 0.0, M[3] = {0, 0, 0};
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                int64_t i = site_index(p, x, y, z);
                int64_t fwd[3] = {site_index(p, x + 1, y, z), site_index(p, x, y + 1, z),
                                  site_index(p, x, y, z + 1)};
                for (int b = 0; b < 3; ++b)
                    if (fwd[b] >= 0)
                        for (int c = 0; c < 3; ++c) bonds += fin[c * N + i] * fin[c * N + fwd[b]];
                sz2 += fin[2 * N + i] * fin[2 * N + i];
                for (int c = 0; c < 3; ++c) {
                    M[c] += fin[c * N + i];
                    /* dL/ds_n = dLdE (-H_eff/N) + dLdM / N */
                    lam[c * N + i] = (-dLdE * Hf[c * N + i] + dLdM[c]) / (double)N;
                    if (gh) gh[c * N + i] += -dLdE * fin[c * N + i] / (double)N;
                }
            }
    /* explicit dependence of E(s_n) on the parameters */
    *gJ += -dLdE * bonds / (double)N;
    *gD += -dLdE * sz2 / (double)N;
    for (int c = 0; c < 3; ++c) gH[c] += -dLdE * M[c] / (double)N;
    for (int64_t m = nsteps; m >= 1; --m) {
        int64_t n = n0 + m;
        int pul = noise && orc_is_pulse_step(n, p->R);
        orc_step_vjp(p, states + (m - 1) * len, hsite, pul, orc_pulse_number(n, p->R), lam, gJ, gD, gH, gh);
    }
    if (gs0) memcpy(gs0, lam, sizeof(double) * len);
    free(states); free(lam); free(Hf);
}
