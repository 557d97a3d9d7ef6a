// C-ABI of the pulse-noise lattice library: handles, parameter validation,
// the pulse/sample schedule of Eq. (ST-expansion), workspace layout and the
// CUDA-graph cache for whole noise intervals.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/spinpulse.h"
#include "spin_internal.h"

using namespace spin;

struct spin_lattice {
    spin_params p;
    Geom g;
    Tableau tab;
    int elt;                 // bytes per real
    void* buf[2][3];         // [0] caller arrays, [1] workspace copy
    const void* hs[3];       // per-site field or nulls
    int cur;                 // which buffer holds the current state
    cudaStream_t st;
    long long n;             // completed steps
    long long eager_intervals;
    // workspace carve-out
    void* tmp;
    double* partials;
    int nblocks_obs;
    double* out_sample;
    double* out_obs;
    long long* d_interval;
    long long* d_sample_count;
    int* d_status;           // bit 0: a bounded device wait gave up
    double* ring;
    long long samples_read;
    cudaGraphExec_t graph[2];  // one noise interval starting from buffer 0 / 1
    cudaStream_t capture_stream;
    // trajectory recording for the adjoint
    bool rec_active;
    int rec_K;
    long long rec_n0, rec_max;
    void* rec_store;
    char err[512];
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t alt[3];
    size_t tmp;
    size_t partials;
    size_t out_sample, out_obs, interval, sample_count, status, ring;
    size_t total;
};

int validate(const spin_params* p) {
    if (!p) return SPIN_EINVAL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return SPIN_EINVAL;
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (N >= (1LL << 31)) return SPIN_EINVAL;
    if (p->precision != 32 && p->precision != 64) return SPIN_EINVAL;
    if (p->integrator < 0 || p->integrator > 3) return SPIN_EINVAL;
    if (p->steps_per_pulse < 1) return SPIN_EINVAL;
    if (!std::isfinite(p->dt) || p->dt == 0.0) return SPIN_EINVAL;
    if (!(p->lambda >= 0.0) || !(p->T >= 0.0) || !std::isfinite(p->lambda) || !std::isfinite(p->T)) return SPIN_EINVAL;
    if (!std::isfinite(p->J) || !std::isfinite(p->D)) return SPIN_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->H[a])) return SPIN_EINVAL;
    if (p->path < 0 || p->path > 1 || p->bc < 0 || p->bc > 1) return SPIN_EINVAL;
    if (p->replica < 0) return SPIN_EINVAL;
    if (p->noise < 0 || p->noise > 2) return SPIN_EINVAL;
    if (p->noise == 2) return SPIN_EUNSUPPORTED;  // rectangular noise: single-spin calls only
    return SPIN_OK;
}

Layout layout_for(const spin_params* p) {
    Layout L{};
    const Geom g{p->nx, p->ny, p->nz};
    const size_t elt = p->precision == 64 ? 8 : 4;
    const size_t comp = align_up(elt * (size_t)g.N());
    size_t off = 0;
    for (int c = 0; c < 3; ++c) {
        L.alt[c] = off;
        off += comp;
    }
    const Tableau tb = tableau_for(p->integrator);
    const bool generic = !tb.chain || p->path == 1 || !(tb.stages == 2 || tb.stages == 4);
    L.tmp = off;
    if (generic) off += align_up(elt * (size_t)(tb.stages + 1) * 3 * (size_t)g.N());
    L.partials = off;
    off += align_up(sizeof(double) * 5 * (size_t)observables_blocks(g));
    L.out_sample = off;
    off += align_up(sizeof(double) * 8);
    L.out_obs = off;
    off += align_up(sizeof(double) * 8);
    L.interval = off;
    off += align_up(sizeof(long long));
    L.sample_count = off;
    off += align_up(sizeof(long long));
    L.status = off;
    off += align_up(sizeof(int));
    L.ring = off;
    off += align_up(sizeof(double) * 5 * SPIN_SAMPLE_RING);
    L.total = off;
    return L;
}

int set_err(spin_lattice* h, int code, const char* fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define SPIN_CUDA(h, call)                                                                          \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return set_err(h, SPIN_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool is_pulse_step(long long n, int R) { return (n % R) == (R / 2); }

template <typename real>
StepLaunch<real> make_launch(spin_lattice* h, int from, bool pulse) {
    StepLaunch<real> L{};
    for (int c = 0; c < 3; ++c) {
        L.in[c] = static_cast<const real*>(h->buf[from][c]);
        L.out[c] = static_cast<real*>(h->buf[from ^ 1][c]);
        L.hs[c] = static_cast<const real*>(h->hs[c]);
    }
    L.g = h->g;
    L.ph.J = (real)h->p.J;
    L.ph.twoD = (real)(2.0 * h->p.D);
    for (int a = 0; a < 3; ++a) L.ph.H[a] = (real)h->p.H[a];
    L.ph.lambda = (real)h->p.lambda;
    L.dt = h->p.dt;
    L.tab = &h->tab;
    L.precession = h->p.precession;
    L.renorm = h->p.renorm;
    L.pulse = pulse ? 1 : 0;
    L.seed = h->p.seed;
    L.replica = (uint64_t)h->p.replica;
    L.sigma = (real)std::sqrt(2.0 * h->p.lambda * h->p.T * h->p.steps_per_pulse * std::fabs(h->p.dt));
    L.d_interval = h->d_interval;
    L.d_status = h->d_status;
    L.tmp = static_cast<real*>(h->tmp);
    L.stream = h->st;
    L.force_generic = h->p.path == 1;
    L.bc = h->p.bc;
    return L;
}

Phys<double> phys64(const spin_lattice* h) {
    Phys<double> ph{};
    ph.J = h->p.J;
    ph.twoD = 2.0 * h->p.D;
    for (int a = 0; a < 3; ++a) ph.H[a] = h->p.H[a];
    ph.lambda = h->p.lambda;
    return ph;
}

// Launch observables of buffer b; sample=true records into the ring.
cudaError_t observe(spin_lattice* h, int b, bool sample, cudaStream_t st) {
    if (h->elt == 4) {
        const float* s[3] = {(const float*)h->buf[b][0], (const float*)h->buf[b][1], (const float*)h->buf[b][2]};
        const float* hs[3] = {(const float*)h->hs[0], (const float*)h->hs[1], (const float*)h->hs[2]};
        return launch_observables<float>(s, hs, h->g, phys64(h), h->partials, h->nblocks_obs,
                                         sample ? h->out_sample : h->out_obs, sample ? h->ring : nullptr,
                                         SPIN_SAMPLE_RING, h->d_interval, h->d_sample_count, h->p.steps_per_pulse, st,
                                         h->p.bc);
    }
    const double* s[3] = {(const double*)h->buf[b][0], (const double*)h->buf[b][1], (const double*)h->buf[b][2]};
    const double* hs[3] = {(const double*)h->hs[0], (const double*)h->hs[1], (const double*)h->hs[2]};
    return launch_observables<double>(s, hs, h->g, phys64(h), h->partials, h->nblocks_obs,
                                      sample ? h->out_sample : h->out_obs, sample ? h->ring : nullptr,
                                      SPIN_SAMPLE_RING, h->d_interval, h->d_sample_count, h->p.steps_per_pulse, st,
                                      h->p.bc);
}

// One step n -> n+1 from buffer `from` on stream st (no host bookkeeping).
cudaError_t launch_one_step(spin_lattice* h, int from, long long n_next, cudaStream_t st) {
    const bool pulse = h->p.noise && is_pulse_step(n_next, h->p.steps_per_pulse);
    cudaError_t e;
    if (h->elt == 4) {
        StepLaunch<float> L = make_launch<float>(h, from, pulse);
        L.stream = st;
        e = launch_step<float>(L);
    } else {
        StepLaunch<double> L = make_launch<double>(h, from, pulse);
        L.stream = st;
        e = launch_step<double>(L);
    }
    if (e != cudaSuccess) return e;
    if (n_next % h->p.steps_per_pulse == 0) e = observe(h, from ^ 1, true, st);
    return e;
}

// Capture one full interval (R steps + sample) starting from buffer `from`.
int capture_interval(spin_lattice* h, int from) {
    if (!h->capture_stream) SPIN_CUDA(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    cudaStream_t cs = h->capture_stream;
    SPIN_CUDA(h, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const int R = h->p.steps_per_pulse;
    int b = from;
    cudaError_t e = cudaSuccess;
    // the graph covers steps mR+1 .. mR+R; pulse and sample positions depend
    // only on n mod R, so step numbers 1..R describe every interval
    for (int q = 1; q <= R && e == cudaSuccess; ++q) {
        e = launch_one_step(h, b, q, cs);
        b ^= 1;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return set_err(h, SPIN_ECUDA, "interval capture: %s", cudaGetErrorString(e));
    }
    if (e2 != cudaSuccess) return set_err(h, SPIN_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
    cudaError_t e3 = cudaGraphInstantiate(&h->graph[from], graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
        h->graph[from] = nullptr;
        return set_err(h, SPIN_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e3));
    }
    return SPIN_OK;
}

// While recording, copy the current state into checkpoint slot (n-n0)/K
// whenever n - n0 is a multiple of K within the recorded range.
int record_if_due(spin_lattice* h) {
    if (!h->rec_active) return SPIN_OK;
    const long long d = h->n - h->rec_n0;
    if (d < 0 || d > h->rec_max || d % h->rec_K != 0) return SPIN_OK;
    const size_t comp = (size_t)h->elt * (size_t)h->g.N();
    char* slot = static_cast<char*>(h->rec_store) + (size_t)(d / h->rec_K) * 3 * comp;
    for (int c = 0; c < 3; ++c)
        SPIN_CUDA(h, cudaMemcpyAsync(slot + c * comp, h->buf[h->cur][c], comp, cudaMemcpyDeviceToDevice, h->st));
    return SPIN_OK;
}

template <typename real>
int backward_t(spin_lattice* h, const double dLdM[3], double dLdE, void* ws, double* gJ, double* gD,
                      double gH[3], void* g_h_site, void* g_s0) {
    AdjointRun<real> A{};
    A.g = h->g;
    A.tab = &h->tab;
    A.K = h->rec_K;
    A.n0 = h->rec_n0;
    A.n_end = h->n;
    A.R = h->p.steps_per_pulse;
    A.noise = h->p.noise;
    A.precession = h->p.precession;
    A.renorm = h->p.renorm;
    A.bc = h->p.bc;
    A.store_stages = adjoint_stores_stages(h->g, (int)sizeof(real), h->tab, h->p.path, h->rec_K) ? 1 : 0;
    A.seed = h->p.seed;
    A.replica = (uint64_t)h->p.replica;
    A.sigma = std::sqrt(2.0 * h->p.lambda * h->p.T * h->p.steps_per_pulse * std::fabs(h->p.dt));
    A.J = h->p.J;
    A.D = h->p.D;
    for (int a = 0; a < 3; ++a) {
        A.H[a] = h->p.H[a];
        A.dLdM[a] = dLdM[a];
    }
    A.lambda = h->p.lambda;
    A.dt = h->p.dt;
    A.h_site = static_cast<const real*>(h->hs[0]);
    A.store = static_cast<const real*>(h->rec_store);
    for (int c = 0; c < 3; ++c) A.final_state[c] = static_cast<const real*>(h->buf[h->cur][c]);
    A.step_template = make_launch<real>(h, 0, false);
    A.workspace = ws;
    A.stream = h->st;
    A.dLdE = dLdE;
    A.gJ = gJ;
    A.gD = gD;
    A.gH = gH;
    A.g_h = static_cast<double*>(g_h_site);
    A.g_s0 = static_cast<real*>(g_s0);
    if (g_h_site) SPIN_CUDA(h, cudaMemsetAsync(g_h_site, 0, sizeof(double) * 3 * (size_t)h->g.N(), h->st));
    SPIN_CUDA(h, adjoint_run<real>(A));
    int status = 0;   // the recomputing steps' bounded waits (adjoint_run has synchronised)
    SPIN_CUDA(h, cudaMemcpy(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status & 1) return set_err(h, SPIN_ETIMEOUT, "a bounded wait in the fused step gave up; the gradients are invalid");
    return SPIN_OK;
}

}  // namespace

extern "C" {

const char* spin_strerror(int status) {
    switch (status) {
        case SPIN_OK: return "ok";
        case SPIN_WARN_APPLICABILITY: return "pulse-noise applicability condition violated (Lambda_N Delta t or lambda H Delta t too large)";
        case SPIN_EINVAL: return "invalid argument";
        case SPIN_ECUDA: return "CUDA runtime error";
        case SPIN_ENONFINITE: return "non-finite spin (integration unstable)";
        case SPIN_ETIMEOUT: return "bounded device wait timed out";
        case SPIN_EUNSUPPORTED: return "unsupported request";
        case SPIN_ENOSPACE: return "workspace too small";
        default: return "unknown status";
    }
}

const char* spin_last_error(const spin_lattice* h) { return h ? h->err : "null handle"; }

int spin_workspace_size(const spin_params* p, size_t* bytes) {
    if (!bytes) return SPIN_EINVAL;
    int v = validate(p);
    if (v != SPIN_OK) return v;
    *bytes = layout_for(p).total;
    return SPIN_OK;
}

int spin_lattice_create(const spin_params* p, void* sx, void* sy, void* sz, const void* h_site, void* workspace,
                        size_t workspace_bytes, void* cuda_stream, spin_lattice** out) {
    if (!out) return SPIN_EINVAL;
    *out = nullptr;
    int v = validate(p);
    if (v != SPIN_OK) return v;
    if (!sx || !sy || !sz || !workspace) return SPIN_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign != 0) return SPIN_EINVAL;
    const Layout L = layout_for(p);
    if (workspace_bytes < L.total) return SPIN_ENOSPACE;

    spin_lattice* h = new (std::nothrow) spin_lattice();
    if (!h) return SPIN_EINVAL;
    h->p = *p;
    h->g = Geom{p->nx, p->ny, p->nz};
    h->tab = tableau_for(p->integrator);
    h->elt = p->precision == 64 ? 8 : 4;
    h->buf[0][0] = sx;
    h->buf[0][1] = sy;
    h->buf[0][2] = sz;
    char* ws = static_cast<char*>(workspace);
    for (int c = 0; c < 3; ++c) h->buf[1][c] = ws + L.alt[c];
    const size_t comp_bytes = (size_t)h->elt * (size_t)h->g.N();
    for (int c = 0; c < 3; ++c) h->hs[c] = h_site ? static_cast<const char*>(h_site) + c * comp_bytes : nullptr;
    h->cur = 0;
    h->st = static_cast<cudaStream_t>(cuda_stream);
    h->n = 0;
    h->tmp = ws + L.tmp;
    h->partials = reinterpret_cast<double*>(ws + L.partials);
    h->nblocks_obs = observables_blocks(h->g);
    h->out_sample = reinterpret_cast<double*>(ws + L.out_sample);
    h->out_obs = reinterpret_cast<double*>(ws + L.out_obs);
    h->d_interval = reinterpret_cast<long long*>(ws + L.interval);
    h->d_sample_count = reinterpret_cast<long long*>(ws + L.sample_count);
    h->d_status = reinterpret_cast<int*>(ws + L.status);
    h->ring = reinterpret_cast<double*>(ws + L.ring);
    h->err[0] = 0;

    cudaError_t e = h->elt == 4 ? prepare_step_kernels<float>() : prepare_step_kernels<double>();
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_interval, 0, sizeof(long long), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_sample_count, 0, sizeof(long long), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st);
    if (e != cudaSuccess) {
        delete h;
        return SPIN_ECUDA;
    }
    *out = h;

    // Applicability of the pulse-noise approximation, Eqs. (phi_condition)
    // and (non-thermal_condition).
    const double Dt = p->steps_per_pulse * std::fabs(p->dt);
    const double LN_Dt = 2.0 * p->lambda * p->T * Dt;
    const double Hmax = 6.0 * std::fabs(p->J) + 2.0 * std::fabs(p->D) +
                        std::sqrt(p->H[0] * p->H[0] + p->H[1] * p->H[1] + p->H[2] * p->H[2]);
    if (p->noise && (LN_Dt > 0.2 || p->lambda * Hmax * Dt > 1.0)) {
        set_err(h, SPIN_WARN_APPLICABILITY, "Lambda_N*Dt = %g, lambda*Hmax*Dt = %g", LN_Dt, p->lambda * Hmax * Dt);
        return SPIN_WARN_APPLICABILITY;
    }
    return SPIN_OK;
}

int spin_step_pulse(spin_lattice* h, int64_t nsteps) {
    if (!h || nsteps < 0) return SPIN_EINVAL;
    const int R = h->p.steps_per_pulse;
    while (nsteps > 0) {
        if (h->rec_active) {
            // recording: a whole noise interval is replayed from the graph when
            // no checkpoint falls strictly inside it (one at its end is taken
            // after the replay); otherwise single eager steps, so that every
            // checkpoint step is seen
            const long long d0 = h->n - h->rec_n0;
            const long long next_ckpt = (d0 / h->rec_K + 1) * h->rec_K;
            if (h->n % R == 0 && nsteps >= R && h->eager_intervals > 0 && d0 >= 0 && next_ckpt >= d0 + R) {
                if (!h->graph[h->cur]) {
                    int rc = capture_interval(h, h->cur);
                    if (rc != SPIN_OK) return rc;
                }
                SPIN_CUDA(h, cudaGraphLaunch(h->graph[h->cur], h->st));
                h->n += R;
                if (R & 1) h->cur ^= 1;
                nsteps -= R;
                int rc = record_if_due(h);
                if (rc != SPIN_OK) return rc;
                continue;
            }
            if (h->n % R == 0 && nsteps >= R) h->eager_intervals++;
            SPIN_CUDA(h, launch_one_step(h, h->cur, h->n + 1, h->st));
            h->cur ^= 1;
            h->n += 1;
            nsteps -= 1;
            int rc = record_if_due(h);
            if (rc != SPIN_OK) return rc;
            continue;
        }
        if (h->n % R == 0 && nsteps >= R && h->eager_intervals > 0) {
            if (!h->graph[h->cur]) {
                int rc = capture_interval(h, h->cur);
                if (rc != SPIN_OK) return rc;
            }
            SPIN_CUDA(h, cudaGraphLaunch(h->graph[h->cur], h->st));
            h->n += R;
            if (R & 1) h->cur ^= 1;
            nsteps -= R;
            continue;
        }
        const bool interval_start = h->n % R == 0 && nsteps >= R;
        const int steps = interval_start ? R : 1;
        for (int q = 0; q < steps; ++q) {
            SPIN_CUDA(h, launch_one_step(h, h->cur, h->n + 1, h->st));
            h->cur ^= 1;
            h->n += 1;
        }
        nsteps -= steps;
        if (interval_start) h->eager_intervals++;
    }
    if (h->cur == 1) {
        const size_t bytes = (size_t)h->elt * (size_t)h->g.N();
        for (int c = 0; c < 3; ++c)
            SPIN_CUDA(h, cudaMemcpyAsync(h->buf[0][c], h->buf[1][c], bytes, cudaMemcpyDeviceToDevice, h->st));
        h->cur = 0;
    }
    return SPIN_OK;
}

int spin_observables(spin_lattice* h, double M[3], double* E) {
    if (!h || !M || !E) return SPIN_EINVAL;
    SPIN_CUDA(h, observe(h, h->cur, false, h->st));
    double o[5];
    int status = 0;
    SPIN_CUDA(h, cudaMemcpyAsync(o, h->out_obs, sizeof(o), cudaMemcpyDeviceToHost, h->st));
    SPIN_CUDA(h, cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    SPIN_CUDA(h, cudaStreamSynchronize(h->st));
    if (status & 1) return set_err(h, SPIN_ETIMEOUT, "a bounded wait in the fused step gave up; the state is invalid");
    M[0] = o[0];
    M[1] = o[1];
    M[2] = o[2];
    *E = o[3];
    if (o[4] != 0.0) return set_err(h, SPIN_ENONFINITE, "%.0f non-finite spins", o[4]);
    return SPIN_OK;
}

int spin_samples(spin_lattice* h, double* out, int64_t max_records, int64_t* count) {
    if (!h || !count || (max_records > 0 && !out) || max_records < 0) return SPIN_EINVAL;
    long long total = 0;
    int status = 0;
    SPIN_CUDA(h, cudaMemcpyAsync(&total, h->d_sample_count, sizeof(total), cudaMemcpyDeviceToHost, h->st));
    SPIN_CUDA(h, cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    SPIN_CUDA(h, cudaStreamSynchronize(h->st));
    if (status & 1) return set_err(h, SPIN_ETIMEOUT, "a bounded wait in the fused step gave up; the state is invalid");
    long long first = h->samples_read;
    if (total - first > SPIN_SAMPLE_RING) first = total - SPIN_SAMPLE_RING;
    if (total - first > max_records) first = total - max_records;
    const long long n = total - first;
    for (long long q = 0; q < n; ++q) {
        const long long slot = (first + q) % SPIN_SAMPLE_RING;
        SPIN_CUDA(h, cudaMemcpyAsync(out + 5 * q, h->ring + 5 * slot, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    }
    SPIN_CUDA(h, cudaStreamSynchronize(h->st));
    h->samples_read = total;
    *count = n;
    return SPIN_OK;
}

int spin_get_step(const spin_lattice* h, int64_t* n) {
    if (!h || !n) return SPIN_EINVAL;
    *n = h->n;
    return SPIN_OK;
}

int spin_set_step(spin_lattice* h, int64_t n) {
    if (!h || n < 0) return SPIN_EINVAL;
    h->n = n;
    SPIN_CUDA(h, launch_set_counter(h->d_interval, n / h->p.steps_per_pulse, h->st));
    return SPIN_OK;
}

int spin_record_store_size(const spin_params* p, int32_t K, int64_t nsteps, size_t* bytes) {
    if (!bytes || K < 1 || nsteps < 1) return SPIN_EINVAL;
    int v = validate(p);
    if (v != SPIN_OK) return v;
    const size_t comp = (size_t)(p->precision == 64 ? 8 : 4) * (size_t)p->nx * p->ny * p->nz;
    *bytes = (size_t)((nsteps + K - 1) / K + 1) * 3 * comp;
    return SPIN_OK;
}

int spin_record_begin(spin_lattice* h, int32_t K, int64_t nsteps, void* store, size_t store_bytes) {
    if (!h || !store || K < 1 || nsteps < 1) return SPIN_EINVAL;
    size_t need = 0;
    spin_record_store_size(&h->p, K, nsteps, &need);
    if (store_bytes < need) return SPIN_ENOSPACE;
    h->rec_active = true;
    h->rec_K = K;
    h->rec_n0 = h->n;
    h->rec_max = nsteps;
    h->rec_store = store;
    return record_if_due(h);
}

int spin_backward_workspace_size(const spin_params* p, int32_t K, size_t* bytes) {
    if (!bytes || K < 1) return SPIN_EINVAL;
    int v = validate(p);
    if (v != SPIN_OK) return v;
    const Tableau tb = tableau_for(p->integrator);
    *bytes = adjoint_workspace_bytes(Geom{p->nx, p->ny, p->nz}, p->precision == 64 ? 8 : 4, tb, p->path, K);
    return SPIN_OK;
}

int spin_backward(spin_lattice* h, const double dLdM[3], double dLdE, void* workspace, size_t workspace_bytes,
                  double* gJ, double* gD, double gH[3], void* g_h_site, void* g_s0) {
    if (!h || !dLdM || !gJ || !gD || !gH || !workspace) return SPIN_EINVAL;
    if (!h->rec_active) return set_err(h, SPIN_EINVAL, "no recorded trajectory (call spin_record_begin first)");
    if (h->n <= h->rec_n0 || h->n - h->rec_n0 > h->rec_max)
        return set_err(h, SPIN_EINVAL, "recorded range %lld..%lld does not end at the current step %lld",
                       h->rec_n0, h->rec_n0 + h->rec_max, h->n);
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign != 0) return SPIN_EINVAL;
    size_t need = 0;
    spin_backward_workspace_size(&h->p, h->rec_K, &need);
    if (workspace_bytes < need) return SPIN_ENOSPACE;
    if (h->elt == 4) return backward_t<float>(h, dLdM, dLdE, workspace, gJ, gD, gH, g_h_site, g_s0);
    return backward_t<double>(h, dLdM, dLdE, workspace, gJ, gD, gH, g_h_site, g_s0);
}

int spin_record_end(spin_lattice* h) {
    if (!h) return SPIN_EINVAL;
    h->rec_active = false;
    return SPIN_OK;
}

int spin_lattice_destroy(spin_lattice* h) {
    if (!h) return SPIN_EINVAL;
    for (int b = 0; b < 2; ++b)
        if (h->graph[b]) cudaGraphExecDestroy(h->graph[b]);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    delete h;
    return SPIN_OK;
}

int spin_noise_draw(uint64_t seed, int64_t k, int64_t replica, int64_t n_sites, int32_t precision, uint64_t* words,
                    void* gauss, void* cuda_stream) {
    if (n_sites < 0 || k < 0 || replica < 0 || (precision != 32 && precision != 64)) return SPIN_EINVAL;
    if (n_sites == 0) return SPIN_OK;
    if (!words && !gauss) return SPIN_EINVAL;
    cudaError_t e = launch_noise_draw(seed, k, replica, n_sites, precision, words, gauss,
                                      static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

}  // extern "C"
