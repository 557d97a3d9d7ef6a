/*
 * spinpulse — GB300 (sm_103a) library for the pulse-noise many-spin time step
 * of D. A. Garanin, "Pulse-noise approach for classical spin systems"
 * (arXiv:1610.04914).
 *
 * The problem (paper Sec. I-II, IV): classical unit spins s_i on a simple-cubic
 * lattice evolve by the Landau-Lifshitz equation, Eq. (LLL),
 *     ds/dt = gamma s x H_eff - gamma lambda s x (s x H_eff)        (noiseless part)
 * integrated with a Runge-Kutta step delta t, the spins renormalised to |s| = 1
 * after each step, and the thermal noise replaced by instantaneous random
 * rotations (Eq. phi_n, Eq. s_rotation) once per interval Delta t = R delta t,
 * placed mid-interval by the Suzuki-Trotter splitting, Eq. (ST-expansion).
 * Units: gamma = mu0 = k_B = 1.
 *
 * Conventions for every entry point below:
 *  - Return value: SPIN_OK (0) on success, a negative spin_status on error,
 *    SPIN_WARN_APPLICABILITY (+1) from create when the paper's applicability
 *    conditions are violated (the handle is still created and usable).
 *    Nothing aborts, throws or traps across this boundary.  spin_strerror()
 *    gives a fixed text per code; spin_last_error() the handle's last detail.
 *  - Spin arrays are structure-of-arrays, one array per component, N = nx*ny*nz
 *    elements each, site index i = x + nx*(y + ny*z) (x fastest), element type
 *    float (precision 32) or double (precision 64), in device memory of the
 *    current CUDA device.  They are OWNED BY THE CALLER and borrowed by the
 *    handle for its whole life; the library updates them in place.
 *  - The workspace is caller-owned device memory of at least
 *    spin_workspace_size() bytes, 256-byte aligned, borrowed for the handle's
 *    life.  The library allocates no device memory of its own.
 *  - A handle is bound to one CUDA stream (cudaStream_t passed as void*; NULL
 *    = legacy default stream).  Calls are asynchronous on that stream unless
 *    stated; a handle must not be used from two host threads at once.
 */
#ifndef SPINPULSE_H
#define SPINPULSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spin_status {
    SPIN_OK = 0,
    SPIN_WARN_APPLICABILITY = 1, /* Eq. (phi_condition) or (non-thermal_condition) violated */
    SPIN_EINVAL = -1,            /* bad argument (size, null pointer, parameter range) */
    SPIN_ECUDA = -2,             /* a CUDA runtime call failed; detail in spin_last_error */
    SPIN_ENONFINITE = -3,        /* a spin became NaN/Inf (integration unstable) */
    SPIN_ETIMEOUT = -4,          /* a bounded device wait gave up */
    SPIN_EUNSUPPORTED = -5,      /* valid request the library does not implement */
    SPIN_ENOSPACE = -6           /* workspace smaller than spin_workspace_size() */
} spin_status;

typedef enum spin_integrator {
    SPIN_RK4 = 0,          /* classical 4-stage Runge-Kutta (paper Appendix names it) */
    SPIN_RK5_BUTCHER = 1,  /* Butcher's 6-stage 5th-order method, paper Appendix */
    SPIN_RK2_MIDPOINT = 2, /* RK2 midpoint, paper Appendix */
    SPIN_HEUN = 3          /* Heun (RK2 trapezoid), paper Appendix */
} spin_integrator;

/* Problem statement of one lattice (paper Sec. II and IV). */
typedef struct spin_params {
    int32_t nx, ny, nz;       /* lattice size, each >= 1 */
    int32_t precision;        /* 32 (float state) or 64 (double state) */
    int32_t integrator;       /* spin_integrator */
    int32_t precession;       /* 1: full Eq. (LLL); 0: slow equation, precession dropped (Sec. II) */
    int32_t steps_per_pulse;  /* R = Delta t / delta t >= 1 */
    int32_t renorm;           /* 1: s <- s/|s| after every step (recommended) */
    int32_t noise;            /* 1: apply the pulses; 0: deterministic (tests);
                                 2: rectangular noise, Eq. (zeta_n): the field
                                 zeta = sqrt(2 lambda T / Delta t) G_k added to
                                 H_eff in the precession term of Eq. (LLL) and
                                 held over each interval of R steps (needs
                                 precession = 1; single-spin calls only, the
                                 lattice and batch calls return
                                 SPIN_EUNSUPPORTED) */
    int32_t replica;          /* replica number, third word of the noise counter */
    int32_t path;             /* 0: fused single-kernel step where the tableau allows
                                 (RK4, RK2 midpoint, Heun), else per-stage kernels;
                                 1: per-stage kernels always (cross-check path) */
    int32_t bc;               /* 0: periodic boundaries; 1: free boundaries (the paper's
                                 particle, Sec. IV): a site on a face has no neighbour
                                 across it; batch replicas and the no-alloc observables
                                 are periodic only */
    double J;                 /* nearest-neighbour exchange; E = -J sum_<ij> s_i.s_j */
    double D;                 /* uniaxial anisotropy along z; E = -D sum s_z^2 */
    double H[3];              /* uniform Zeeman field; E = -sum H.s */
    double lambda;            /* dimensionless damping of Eq. (LLL) */
    double T;                 /* temperature (k_B = 1) */
    double dt;                /* integration step delta t */
    uint64_t seed;            /* key of the counter-based noise generator */
} spin_params;

typedef struct spin_lattice spin_lattice;

/*
 * Bytes of workspace a handle for *p needs.  Layout (internal): a second state
 * buffer for the out-of-place stencil update, stage temporaries for
 * multi-kernel integrators, FP64 reduction partials, the device-resident
 * interval counter and the sample ring.
 * Errors: SPIN_EINVAL for a null pointer or invalid parameters.
 */
int spin_workspace_size(const spin_params* p, size_t* bytes);

/*
 * Create a handle for the lattice problem *p (Sec. II, IV).
 *   sx, sy, sz  device arrays of N elements (float or double per p->precision):
 *               the initial spins, unit length; updated in place by later calls.
 *   h_site      nullable: device array of 3N elements (same type), the per-site
 *               field h_i added to H_eff (component-major: x block, y, z).
 *   workspace   device memory of workspace_bytes >= spin_workspace_size(p).
 *   cuda_stream cudaStream_t all work is ordered on.
 * On success *out receives the handle (host memory owned by the library,
 * released by spin_lattice_destroy).  Returns SPIN_WARN_APPLICABILITY when
 * Lambda_N Delta t = 2 lambda T Delta t > 0.2 (Eq. phi_condition) or
 * lambda |H_eff|max Delta t > 1 (Eq. non-thermal_condition).
 * Errors: SPIN_EINVAL (null arrays/out, sizes < 1, N >= 2^31, precision not
 * 32/64, R < 1, dt not finite/zero, lambda or T < 0), SPIN_ENOSPACE, SPIN_ECUDA.
 */
int spin_lattice_create(const spin_params* p, void* sx, void* sy, void* sz,
                        const void* h_site, void* workspace, size_t workspace_bytes,
                        void* cuda_stream, spin_lattice** out);

/*
 * Advance nsteps >= 0 integration steps delta t (asynchronous on the stream).
 * Steps are numbered n = 1, 2, ... over the handle's life.  After step n:
 * the pulse number floor((n-1)/R) is applied when n mod R == floor(R/2)
 * (Eq. ST-expansion: mid-interval; every step when R = 1), and the
 * observables are sampled into the sample ring when n mod R == 0 (Sec. III.A:
 * values at the end of each Delta t).  Full intervals are replayed from a
 * cached CUDA graph.  On return (stream-ordered) the caller's arrays hold the
 * state after the last step.
 * Kernel choice for FP32 RK4 steps (all give bitwise the same states): the
 * register-ring fused step, or, where its wave-cost estimate is lower (large
 * lattices, no per-site field), the step that keeps its older planes in
 * tensor memory; the environment variable SPIN_TMEM=0 / =1, read when a step
 * is launched or captured, forbids / forces the latter, and SPIN_TMA=1
 * stages the spin planes by tensor-map bulk copies instead of cp.async
 * (slower on GB300; kept for measurement).
 * Errors: SPIN_EINVAL (null handle, nsteps < 0), SPIN_ECUDA.
 */
int spin_step_pulse(spin_lattice* h, int64_t nsteps);

/*
 * Observables of the current state, FP64 (Sec. III.A, Sec. IV):
 *   M = (1/N) sum_i s_i,
 *   E = (1/N) [ -J sum_<ij> s_i.s_j - D sum_i s_iz^2 - sum_i (H + h_i).s_i ],
 * each nearest-neighbour bond counted once.  Synchronises the stream.
 * M (3 doubles) and E are host pointers.
 * Errors: SPIN_EINVAL (null pointers), SPIN_ENONFINITE (some spin is NaN/Inf;
 * M and E are still written), SPIN_ECUDA.
 */
int spin_observables(spin_lattice* h, double M[3], double* E);

/*
 * Copy the sample ring to host memory: records of 5 doubles
 * (n, M_x, M_y, M_z, E), oldest first, at most max_records of the newest
 * samples taken since the last call; *count receives the number written.
 * The ring holds SPIN_SAMPLE_RING records; older unread samples are dropped.
 * Synchronises the stream.  Errors: SPIN_EINVAL, SPIN_ECUDA.
 */
#define SPIN_SAMPLE_RING 4096
int spin_samples(spin_lattice* h, double* out, int64_t max_records, int64_t* count);

/* Completed step count n of the handle (host value, no synchronisation). */
int spin_get_step(const spin_lattice* h, int64_t* n);

/*
 * Set the completed step count to n >= 0, e.g. after restoring the spin
 * arrays from a checkpoint: the noise is a pure function of (seed, site,
 * pulse number, replica), so a resumed run reproduces an uninterrupted one
 * bit for bit.  Asynchronous.  Errors: SPIN_EINVAL, SPIN_ECUDA.
 */
int spin_set_step(spin_lattice* h, int64_t n);

/*
 * Trajectory recording for the adjoint (checkpointing).  From the handle's
 * current step n0, spin_step_pulse copies the state into `store` every K steps
 * (slot c holds the state after step n0 + c*K, component-major: 3N values of
 * the state type), for at most nsteps steps; while recording, steps launch one
 * by one (no graph replay).  store: caller-owned device memory of at least
 * spin_record_store_size() bytes, borrowed until spin_record_end.
 * Errors: SPIN_EINVAL (K < 1, nsteps < 1, null), SPIN_ENOSPACE, SPIN_ECUDA.
 */
int spin_record_store_size(const spin_params* p, int32_t K, int64_t nsteps, size_t* bytes);
int spin_record_begin(spin_lattice* h, int32_t K, int64_t nsteps, void* store, size_t store_bytes);
int spin_record_end(spin_lattice* h);

/*
 * Pathwise gradients (noise fixed) of L = dLdE E(s_n) + dLdM . M(s_n) for the
 * recorded run n0 -> n (the current step), E and M per spin as in
 * spin_observables.  This is the discrete adjoint of the whole step: RK
 * stages of Eq. (LLL) (tableaus of the paper's Appendix), renormalisation and
 * the pulse rotation of Eq. (s_rotation) (transposed: rotation by -phi).
 * The backward pass restores each checkpoint, recomputes its K steps with
 * the forward kernels and runs the transposed steps backwards.  For FP32
 * states with a chain tableau (RK4, RK2 midpoint, Heun) on the fused path the
 * recomputing steps also write every stage's input and increment, which the
 * transposed steps read instead of recomputing them; the workspace then holds
 * (2 x stages - 1) x K extra arrays of 3N values (taken only while they come
 * to at most 8 GiB; otherwise the stages are recomputed per step).
 *   dLdM, dLdE   host seeds of the loss
 *   workspace    device, >= spin_backward_workspace_size(p, K) bytes, 256-aligned
 *   gJ, gD, gH   host outputs: dL/dJ, dL/dD, dL/dH (3), including the explicit
 *                dependence of E(s_n) on the parameters
 *   g_h_site     nullable device FP64 array of 3N: dL/dh_i (component-major)
 *   g_s0         nullable device array of 3N (state type): dL/ds_{n0}
 * Parameter gradients accumulate in FP64: every site's term of every stage of
 * every step is formed in the state precision and added in FP64 (dL/dh_i
 * straight into g_h_site; dL/dJ, dL/dD, dL/dH through FP64 per-thread sums
 * reduced in FP64).  The adjoint state is kept in the state precision.
 * Synchronises the stream.
 * Errors: SPIN_EINVAL (no recording, range mismatch), SPIN_ENOSPACE, SPIN_ECUDA.
 */
int spin_backward_workspace_size(const spin_params* p, int32_t K, size_t* bytes);
int spin_backward(spin_lattice* h, const double dLdM[3], double dLdE, void* workspace,
                  size_t workspace_bytes, double* gJ, double* gD, double gH[3], void* g_h_site,
                  void* g_s0);

/* Release the handle's host state and CUDA graphs (not the borrowed arrays). */
int spin_lattice_destroy(spin_lattice* h);

const char* spin_strerror(int status);
const char* spin_last_error(const spin_lattice* h);

/*
 * The noise draw of Eq. (phi_n) on its own, for verification: for sites
 * i = 0..n_sites-1 computes the four Philox4x64-10 words of counter
 * (i, k, replica, 0) under key (seed, noise stream) into words[4*i+0..3]
 * (device, uint64) and, if gauss is non-null, the Box-Muller normals
 * G_i (device, 3*n_sites, component-minor: gauss[3*i+a]) in the given
 * precision (32: float, 64: double).  Asynchronous on cuda_stream.
 * Errors: SPIN_EINVAL, SPIN_ECUDA.
 */
int spin_noise_draw(uint64_t seed, int64_t k, int64_t replica, int64_t n_sites,
                    int32_t precision, uint64_t* words, void* gauss, void* cuda_stream);

/*
 * Batched replicas: nrep independent cubic periodic lattices of sides L[r]
 * and temperatures T[r] (the paper's ensemble runs "in parallel cycles",
 * Sec. III.A and Appendix), advanced together by one kernel launch per step
 * over a table of (replica, tile, z-chunk) work items.  All replicas share
 * the other spin_params fields (J, D, H, lambda, dt, R, integrator, seed;
 * nx, ny, nz, replica and path are ignored); replica r draws its noise with
 * counter word 2 = r, so replica r of a batch reproduces a single lattice
 * created with replica = r.  FP32 state and chain tableaus (RK4, RK2
 * midpoint, Heun) only; other requests return SPIN_EUNSUPPORTED.
 *
 * State: three caller-owned device float arrays (s_x, s_y, s_z) holding the
 * replicas back to back, replica r at offset offsets[r] (spin_batch_offsets:
 * offsets[r] = sum_{q<r} L[q]^3, offsets[nrep] = total), each replica x
 * fastest.
 * Tiling: chosen per size class (the replicas sharing one side L) as a CTA
 * tile height tile_rows (spin_batch_tile_rows lists the heights offered for
 * an integrator; a tile writes tile_rows - 2 x stages rows, the rest is the
 * stage halo) and a z-chunk length chunk (planes per work item, >= 1).  It
 * changes the schedule only: every tiling gives bit-identical states.
 * chunk_planes at create: > 0 gives every class that chunk and the tallest
 * tile; -1 gives every class the default (tallest tile, chunk 32) without
 * timing; 0 autotunes: per class, in decreasing order of spins, each tile
 * height x chunk in {8, 16, 32, 64} is timed on the whole batch (one step,
 * input buffer to scratch, state untouched; synchronous) with the other
 * classes held, and the fastest kept.  Classes tuned earlier in the process
 * for the same (L, precision, integrator) reuse that choice.
 * spin_batch_tiling reports the per-class choice; spin_batch_set_tiling pins
 * the listed classes (SPIN_EINVAL for a side no replica has, a height not
 * offered, or chunk < 1); spin_batch_autotune tunes the classes not pinned.
 * Both synchronise the stream and rebuild the work-item table.
 * Samples: after steps with n mod R == 0 a record of nrep x 5 doubles
 * (n, M_x, M_y, M_z, E per replica) goes to a ring of
 * SPIN_BATCH_SAMPLE_RING records.
 * Errors as for the single-lattice calls.
 */
#define SPIN_BATCH_SAMPLE_RING 512
typedef struct spin_batch spin_batch;
int spin_batch_offsets(int32_t nrep, const int32_t* L, int64_t* offsets);
int spin_batch_workspace_size(const spin_params* p, int32_t nrep, const int32_t* L, size_t* bytes);
int spin_batch_create(const spin_params* p, int32_t nrep, const int32_t* L, const double* T, void* sx,
                      void* sy, void* sz, int32_t chunk_planes, void* workspace, size_t workspace_bytes,
                      void* cuda_stream, spin_batch** out);
/* chunk of the class holding the most spins, and the number of work items */
int spin_batch_tuning(const spin_batch* b, int32_t* chunk_planes, int32_t* nitems);
/* tile heights offered for integrator (the tallest first) into rows[max]; *n = their count */
int spin_batch_tile_rows(int32_t integrator, int32_t max, int32_t* rows, int32_t* n);
/* per size class (first-appearance order): side, tile height, chunk into arrays of max entries; *n = classes */
int spin_batch_tiling(const spin_batch* b, int32_t max, int32_t* L, int32_t* tile_rows, int32_t* chunk,
                      int32_t* n);
int spin_batch_set_tiling(spin_batch* b, int32_t n, const int32_t* L, const int32_t* tile_rows,
                          const int32_t* chunk);
int spin_batch_autotune(spin_batch* b);
int spin_batch_step_pulse(spin_batch* b, int64_t nsteps);
/* current M_x, M_y, M_z, E, non-finite count per replica into host out[5*nrep]; synchronises */
int spin_batch_observables(spin_batch* b, double* out);
/* up to max_records unread sample records into host out[max_records*nrep*5]; synchronises */
int spin_batch_samples(spin_batch* b, double* out, int64_t max_records, int64_t* count);
int spin_batch_destroy(spin_batch* b);
const char* spin_batch_last_error(const spin_batch* b);

/*
 * Single-spin replicas (paper Sec. III: a spin in a field, Eq. s_evolution_anal,
 * Figs. 1, 2 and 4; a uniaxial spin in a transverse field and its thermally
 * activated escape, Sec. III.B and Fig. 6).  nrep independent spins with
 * energy E = -D s_z^2 - H.s (H_eff = H + 2D s_z z; J, nx, ny, nz, replica,
 * path and bc of p are ignored), one GPU thread each, with the integrator
 * and renormalisation of spin_step_pulse and the noise p->noise: 1 pulses
 * (Eqs. (phi_n), (s_rotation)) after step n with n mod R == R/2, or 2
 * rectangular noise (Eq. (zeta_n)): the field of interval k = (n-1) div R,
 * drawn with the counter of pulse k, added to H_eff in the precession term
 * of every stage of the interval's steps (needs p->precession = 1).
 *   s        device array of 3*nrep values of the state type: s_x of all
 *            replicas, then s_y, then s_z; updated in place
 *   scratch  device array of 2*nrep values of the state type, caller-owned,
 *            filled by spin_single_prepare
 * Errors: SPIN_EINVAL (bad sizes, pointers or parameters), SPIN_ECUDA.
 */

/*
 * spin_single_prepare: replica r has temperature T[r] and damping lambda[r]
 * (host arrays of nrep values; lambda NULL: p->lambda for all).  Computes in
 * FP64 the noise scale of each replica -- sqrt(2 lambda T Delta t) for
 * pulses, sqrt(2 lambda T / Delta t) for rectangular noise, Delta t = R|dt|
 * -- and copies scales and dampings into scratch, synchronously on
 * cuda_stream.  Call again whenever T, lambda, R, dt or the noise kind
 * change; the run and escape calls below read scratch only.
 * Errors: SPIN_EINVAL (also T or lambda negative or non-finite).
 */
int spin_single_prepare(const spin_params* p, int32_t nrep, const double* T, const double* lambda,
                        void* scratch, void* cuda_stream);

/*
 * spin_single_run: advance every replica from completed step n0 by nsteps
 * steps (one kernel launch on cuda_stream, asynchronous); the noise of
 * replica r uses counter (0, k, r, 0), so replica r follows exactly a
 * one-site lattice with replica index r and J = 0.
 *   stop_on_crossing  1: a replica stops after the first step that leaves
 *            s_z < 0 and stores that step number in first_passage[r]
 *            (device int64, -1 = none yet; replicas with a stored step are
 *            skipped by later calls) -- the first-passage procedure of
 *            Sec. III.B
 *   sz_sum, sz_count  nullable device arrays (FP64, int64) accumulating s_z
 *            after every step with n mod R == 0 (equilibrium averages)
 */
int spin_single_run(const spin_params* p, int32_t nrep, void* s, void* scratch, int64_t n0, int64_t nsteps,
                    int32_t stop_on_crossing, int64_t* first_passage, double* sz_sum, int64_t* sz_count,
                    void* cuda_stream);

/*
 * spin_single_escape: renewal form of the first-passage procedure (one
 * kernel launch on cuda_stream, asynchronous).  Every replica advances
 * nsteps steps from completed global step n0.  When a step leaves s_z < 0
 * the replica adds the number of steps of its current trial to fpt_sum[r]
 * (and its square to fpt_sq[r], nullable), increments fpt_count[r] and
 * trial[r], sets local_step[r] = -1 and waits until the next global step n
 * with n mod R == 0 (at most R-1 steps); there it restarts from s_init (host,
 * 3 values, s_init[2] >= 0) with local_step[r] = 0.  Every trial thus starts
 * at the beginning of a noise interval and sees the schedule of a fresh run;
 * trial j of replica r uses noise counter (0, k, r + j*nrep, 0), k counted
 * from the trial's start.  trial, local_step, fpt_sum, fpt_count: device
 * int64 arrays of nrep values.  Start: all zero, s = s_init, n0 = 0 (or any
 * multiple of R); later calls pass n0 = steps completed so far.  A running
 * replica whose local_step is out of phase with n0 (local_step mod R !=
 * n0 mod R) is treated as waiting.  The mean first-passage time is
 * sum(fpt_sum)/sum(fpt_count) steps.
 */
int spin_single_escape(const spin_params* p, int32_t nrep, const double* s_init, void* s, void* scratch,
                       int64_t n0, int64_t nsteps, int64_t* trial, int64_t* local_step, int64_t* fpt_sum,
                       double* fpt_sq, int64_t* fpt_count, void* cuda_stream);

/*
 * Checkerboard Metropolis Monte Carlo (Sec. IV), the paper's comparison
 * method.  nsweeps sweeps numbered sweep0, sweep0+1, ... of the lattice p
 * (J, D, H, T, bc, replica, precision; the dynamics fields are ignored), on
 * the caller's state s (device, SoA, 3N values of the state type, x fastest)
 * and optional per-site field h_site (device, same layout, nullable).  Each
 * sweep first tries every site with x+y+z even, then every site with x+y+z
 * odd (one launch each, asynchronous on cuda_stream).  Trial at site i in
 * sweep w: u uniform on the sphere from Philox4x64-10, counter
 * (i, w, replica, 0), key (mc_seed, 0x6D6F6E7465 "monte"), cos(theta) =
 * 2 u0 - 1, phi = 2 pi u1 with u = ((word >> 11) + 1/2) 2^-53;
 * s' = (s + R_trial u)/|s + R_trial u|; accepted if dE <= 0 or
 * u2 < exp(-dE/T), with dE the change of -s.(J sum_nn s_j + H + h_i) - D s_z^2.
 * R_trial <= 0 selects the paper's 1.55 sqrt(T/(6J)) (needs J > 0).
 * accepted: nullable device int64, incremented by the number of accepted
 * trials.  Periodic lattices need even nx, ny, nz.
 * Errors: SPIN_EINVAL, SPIN_ECUDA.
 */
int spin_metropolis_sweeps(const spin_params* p, void* s, const void* h_site, uint64_t mc_seed, double R_trial,
                           int64_t sweep0, int64_t nsweeps, int64_t* accepted, void* cuda_stream);

/*
 * spin_metropolis_color: one half of sweep `sweep` -- the trials of the
 * sites with (x+y+z) mod 2 == color (0 or 1) only, as spin_metropolis_sweeps
 * does them; colour 0 then colour 1 of the same sweep equal one sweep.
 */
int spin_metropolis_color(const spin_params* p, void* s, const void* h_site, uint64_t mc_seed, double R_trial,
                          int64_t sweep, int32_t color, int64_t* accepted, void* cuda_stream);

/*
 * Observables of caller-owned spin arrays with no memory allocation at all.
 * The paper has no counterpart: this entry point serves callers that cannot
 * call cudaMalloc or ask their framework for memory where they need M and E
 * (a fixed memory budget, a thread that must not enter the allocator, a
 * plug-in that is handed only existing arrays).  It computes the same FP64
 * values as spin_observables without a handle or workspace:
 *   precision   32 (float arrays) or 64 (double arrays)
 *   sx, sy, sz  device arrays of N = nx*ny*nz elements (x fastest)
 *   h_site      nullable, device array of 3N elements (x block, y, z)
 *   J, D, H     as in spin_params (H: host array of 3 doubles)
 *   bc          0 periodic, 1 free boundaries (no bond across a face), as
 *               spin_params.bc
 *   out5        DEVICE array of 5 doubles receiving (M_x, M_y, M_z, E, number
 *               of non-finite spins); written asynchronously on cuda_stream.
 * Scratch: one 5-double record per reduction block lives in a file-scope
 * __device__ array of SPIN_NOALLOC_MAX_BLOCKS records (40 KiB); every GPU that
 * loads the library holds it until the process exits.  All calls share it and
 * it keeps the last call's contents; each call overwrites every record it
 * reads, so nothing needs clearing, but calls that overlap on the GPU (two
 * streams, or two host threads) race on it and must be serialised.  Outside
 * stream capture every call looks up the array's device address on the
 * current device; a call on a stream that is being captured reuses the
 * address that the last uncaptured call on that device found, so make one
 * uncaptured call on each device before capturing one.  cudaDeviceReset
 * reloads the library's module, so after it make one uncaptured call again
 * before any capture.  Lattices of more than SPIN_NOALLOC_MAX_SITES sites are
 * rejected with SPIN_EINVAL.
 * Errors: SPIN_EINVAL (null pointers, precision, bc, sizes < 1 or beyond the
 * maximum, a capture before any uncaptured call on the device), SPIN_ECUDA.
 */
#define SPIN_NOALLOC_MAX_BLOCKS 1024
#define SPIN_NOALLOC_MAX_SITES 2147483647LL
int spin_observables_noalloc(int32_t precision, const void* sx, const void* sy, const void* sz,
                             const void* h_site, int32_t nx, int32_t ny, int32_t nz, double J,
                             double D, const double H[3], int32_t bc, double* out5, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SPINPULSE_H */
