// Internal interfaces between the library's translation units (host side).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace spin {

// Geometry of the lattice: periodic nx*ny*nz, site i = x + nx*(y + ny*z).
struct Geom {
    int nx, ny, nz;
    long long N() const { return (long long)nx * ny * nz; }
};

// Coefficients of one explicit Runge-Kutta tableau (paper Appendix), with
// K_j = dt f(x_j), x_1 = s, x_j = s + sum_{l<j} a[j][l] K_l,
// s' = s + sum_j b[j] K_j.
struct Tableau {
    int stages;
    double a[6][6];
    double b[6];
    bool chain;  // a[j][l] == 0 unless l == j-1: stage j needs only K_{j-1}
};
Tableau tableau_for(int integrator);

// Physical parameters as seen by the kernels.
template <typename real>
struct Phys {
    real J, twoD, H[3], lambda;
};

// Arguments of one step launch.
template <typename real>
struct StepLaunch {
    const real* in[3];
    real* out[3];
    const real* hs[3];     // per-site field or nulls
    Geom g;
    Phys<real> ph;
    double dt;
    const Tableau* tab;
    int precession;
    int renorm;
    int pulse;             // apply the pulse after this step
    uint64_t seed;
    uint64_t replica;
    real sigma;            // pulse angle scale sqrt(2 lambda T Delta t)
    const long long* d_interval;  // device: pulse number of the current interval
    int* d_status;         // device status word (bit 0: a bounded wait in a kernel gave up) or null
    real* tmp;             // generic path: (stages + 1) * 3N scratch
    cudaStream_t stream;
    int force_generic;
    int bc;                // 0 periodic, 1 free boundaries
    // FP32 fused path only: if st_n[0][0] is set, the step also writes, at
    // every site, the stage inputs X_j (j = 2..S, st_x[j-2]), the neighbour
    // sums sum_nn X_j of every stage (j = 1..S, st_n[j-1]) and the
    // unnormalised RK result y (st_y), component arrays of 3 x N
    real* st_x[3][3];
    real* st_n[4][3];
    real* st_y[3];
};

template <typename real>
cudaError_t launch_step(const StepLaunch<real>& L);
// Set the dynamic shared-memory limits of every fused-step instantiation
// (call once per device before launching or capturing).
template <typename real>
cudaError_t prepare_step_kernels();
// FP32 fused step with register patches (chain tableaus, 2 or 4 stages).
cudaError_t launch_step_patch(const StepLaunch<float>& L);
cudaError_t prepare_patch_kernels();
// The noise rotation of Eq. (s_rotation) over every site of L.out, in place.
cudaError_t launch_pulse_lattice(const StepLaunch<float>& L);
// FP32 fused six-stage (Butcher RK5) step in two three-stage segments; needs
// L.tmp with 12N floats (the four carried vectors) and no per-site field.
bool rk5_fused_supports(const StepLaunch<float>& L);
cudaError_t launch_step_rk5(const StepLaunch<float>& L);
cudaError_t prepare_rk5_kernels();
int patch_out_x(int stages);                // output columns per CTA tile along x
int patch_out_y(int stages, int variant);   // ... along y, for tile variant 0 .. patch_variants()-1
int patch_rows(int stages, int variant);    // tile rows (output rows + 2 x stages)
int patch_variants();

// Batched replicas (cubic periodic lattices, one concatenated SoA state).
struct BatchItem {
    int rep;
    short bx, by;
    int bz;
};
struct BatchRep {
    long long off;   // first site of the replica in the concatenated arrays
    int L;           // side
    int tz;          // z chunk (planes)
    float sigma;     // pulse angle scale sqrt(2 lambda T_r Delta t)
    int pad;
};
cudaError_t launch_step_patch_batch(const StepLaunch<float>& L, const BatchItem* items, int nitems,
                                    const BatchRep* reps, int variant);

// Batched observables: block b reduces rows [row0, row0+nrows) of replica rep;
// blocks of one replica are contiguous; first_block has nrep+1 entries.
struct ObsBlock {
    int rep;
    int row0;
    int nrows;
};
// Pulse rotation of every site of every replica (block table as above).
cudaError_t launch_pulse_batch(float* s[3], const BatchRep* reps, const ObsBlock* blocks, int nblocks, uint64_t seed,
                               const long long* d_interval, cudaStream_t st);
cudaError_t launch_observables_batch(const float* s[3], const BatchRep* reps, const ObsBlock* blocks, int nblocks,
                                     const int* first_block, int nrep, Phys<double> ph, double* partials,
                                     double* out, double* ring, int ring_len, long long* d_interval,
                                     long long* d_sample_count, int R, cudaStream_t stream);

// FP64 observables: per-block partials, then a one-block deterministic sum.
// out5 = (M_x, M_y, M_z, E, nonfinite count); if sample_ring != null the
// record (n, M, E) goes to sample_ring[(*d_interval) % ring] with
// n = ((*d_interval) + 1) * R, and *d_interval is incremented.
template <typename real>
cudaError_t launch_observables(const real* s[3], const real* hs[3], Geom g, Phys<double> ph,
                               double* partials, int nblocks, double* out5, double* sample_ring,
                               int ring, long long* d_interval, long long* d_sample_count, int R,
                               cudaStream_t stream, int bc = 0);
int observables_blocks(Geom g);

cudaError_t launch_noise_draw(uint64_t seed, long long k, long long replica, long long n, int precision,
                              uint64_t* words, void* gauss, cudaStream_t stream);

cudaError_t launch_set_counter(long long* d, long long value, cudaStream_t stream);

// Checkpointed discrete adjoint of a recorded run (adjoint.cu).
template <typename real>
struct AdjointRun {
    Geom g;
    const Tableau* tab;
    int K;                   // checkpoint interval (steps)
    long long n0, n_end;     // recorded range: states n0 .. n_end
    int R, noise, precession, renorm, bc;
    int store_stages;        // stage storage of the segment (adjoint_stores_stages)
    uint64_t seed, replica;
    double sigma, J, D, H[3], lambda, dt;
    const real* h_site;      // component-major 3N or null
    const real* store;       // checkpoints: state at n0 + c*K, component-major 3N each
    const real* final_state[3];
    StepLaunch<real> step_template;  // forward kernels for the recomputation
    void* workspace;
    cudaStream_t stream;
    double dLdM[3];
    double dLdE;
    double* gJ;
    double* gD;
    double* gH;              // 3 doubles (host)
    double* g_h;             // device FP64 3N or null
    real* g_s0;              // device 3N or null
};
// Whether the adjoint keeps each checkpoint segment's stage inputs and
// increments from the recomputation (FP32 fused-step path, chain tableaus of 2
// or 4 stages, at most 8 GiB of stage storage) instead of recomputing the
// stages in every transposed step.
bool adjoint_stores_stages(const Geom& g, int elt, const Tableau& tb, int path, int K);
size_t adjoint_workspace_bytes(const Geom& g, int elt, const Tableau& tb, int path, int K);
template <typename real>
cudaError_t adjoint_run(const AdjointRun<real>& A);

}  // namespace spin
