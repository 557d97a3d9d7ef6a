// C-ABI of the batched replicas: many independent cubic periodic lattices of
// uneven size and temperature (the paper's ensemble averaging in "parallel
// cycles", Sec. III.A and the Appendix, done as one GPU launch per step).
// All replicas share J, D, H, lambda, dt, R and the integrator; each has its
// own side L_r, temperature T_r (pulse angle sqrt(2 lambda T_r Delta t)) and
// noise stream (replica index r in the counter).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/spinpulse.h"
#include "spin_internal.h"

using namespace spin;

struct spin_batch {
    spin_params p;
    Tableau tab;
    int nrep;
    std::vector<int> L;
    std::vector<double> T;
    std::vector<int64_t> off;
    long long ntot;
    void* buf[2][3];
    int cur;
    cudaStream_t st;
    long long n;
    long long eager_intervals;
    // device tables in the workspace
    BatchRep* reps;
    BatchItem* items;
    int nitems;
    // tiling per size class (all replicas of one side L): CTA tile variant,
    // z-chunk target, and whether the caller pinned it (autotune skips those)
    std::vector<int> cls_L, cls_var, cls_chunk, cls_pinned;
    std::vector<int> var_first;   // items of tile variant v: [var_first[v], var_first[v+1])
    ObsBlock* oblocks;
    int* first_block;
    int nblocks_obs;
    double* partials;
    double* out;
    long long* d_interval;
    int* d_status;           // bit 0: a bounded device wait gave up
    long long* d_sample_count;
    double* ring;
    long long samples_read;
    cudaGraphExec_t graph[2];
    cudaStream_t capture_stream;
    std::vector<BatchItem> host_items;
    std::vector<BatchRep> host_reps;
    char err[512];
};

namespace {

constexpr size_t kAlign = 256;
size_t al(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr int kRowsPerObsBlock = 256;
const int kChunkCandidates[] = {8, 16, 32, 64};
constexpr int kDefaultChunk = 32;

int bset_err(spin_batch* b, int code, const char* fmt, ...) {
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define BATCH_CUDA(b, call)                                                                           \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return bset_err(b, SPIN_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int validate_batch(const spin_params* p, int nrep, const int32_t* L, const double* T) {
    if (!p || nrep < 1 || !L) return SPIN_EINVAL;
    if (p->noise < 0 || p->noise > 2) return SPIN_EINVAL;
    if (p->precision != 32 || p->bc != 0 || p->noise == 2) return SPIN_EUNSUPPORTED;
    const Tableau tb = tableau_for(p->integrator);
    if (!tb.chain || !(tb.stages == 2 || tb.stages == 4)) return SPIN_EUNSUPPORTED;
    if (p->steps_per_pulse < 1 || !std::isfinite(p->dt) || p->dt == 0.0 || !(p->lambda >= 0.0)) return SPIN_EINVAL;
    long long tot = 0;
    for (int r = 0; r < nrep; ++r) {
        if (L[r] < 1 || L[r] > 1024) return SPIN_EINVAL;
        tot += (long long)L[r] * L[r] * L[r];
        if (T && !(T[r] >= 0.0)) return SPIN_EINVAL;
    }
    if (tot >= (1LL << 31)) return SPIN_EINVAL;
    return SPIN_OK;
}

// Work items of every replica under its class's tiling, grouped by tile
// variant (one launch each); within a variant the most expensive items come
// first, so the block scheduler balances the tail.
std::vector<BatchItem> make_items(const spin_params* p, int nrep, const int32_t* L, const std::vector<int>& var_of,
                                  const std::vector<int>& chunk_of, std::vector<int>* tz_out,
                                  std::vector<int>* var_first) {
    const int S = tableau_for(p->integrator).stages;
    const int nv = patch_variants();
    const int ox = patch_out_x(S);
    std::vector<BatchItem> items;
    tz_out->assign(nrep, 1);
    var_first->assign(nv + 1, 0);
    for (int v = 0; v < nv; ++v) {
        (*var_first)[v] = (int)items.size();
        const int oy = patch_out_y(S, v);
        std::vector<std::pair<int, BatchItem>> w;
        for (int r = 0; r < nrep; ++r) {
            if (var_of[r] != v) continue;
            const int chunks = std::max(1, (L[r] + chunk_of[r] - 1) / chunk_of[r]);
            const int tz = (L[r] + chunks - 1) / chunks;
            (*tz_out)[r] = tz;
            const int tx = (L[r] + ox - 1) / ox, ty = (L[r] + oy - 1) / oy;
            const int used = (L[r] + tz - 1) / tz;
            for (int bz = 0; bz < used; ++bz)
                for (int by = 0; by < ty; ++by)
                    for (int bx = 0; bx < tx; ++bx)
                        w.push_back({tz + 2 * S - 2, BatchItem{r, (short)bx, (short)by, bz}});
        }
        std::stable_sort(w.begin(), w.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
        for (auto& e : w) items.push_back(e.second);
    }
    (*var_first)[nv] = (int)items.size();
    return items;
}

// Largest item table any tiling can produce: per replica, the most items
// over tile variants and z-chunks of at least the smallest candidate.
int max_items(const spin_params* p, int nrep, const int32_t* L) {
    const int S = tableau_for(p->integrator).stages;
    const int ox = patch_out_x(S);
    long long m = 0;
    for (int r = 0; r < nrep; ++r) {
        long long best = 0;
        for (int v = 0; v < patch_variants(); ++v) {
            const int oy = patch_out_y(S, v);
            const long long t = (long long)((L[r] + ox - 1) / ox) * ((L[r] + oy - 1) / oy) * L[r];
            best = std::max(best, t);
        }
        m += best;
    }
    return (int)std::min<long long>(m, 1LL << 30);
}

int obs_blocks(int nrep, const int32_t* L, std::vector<ObsBlock>* blocks, std::vector<int>* first) {
    blocks->clear();
    first->assign(nrep + 1, 0);
    for (int r = 0; r < nrep; ++r) {
        (*first)[r] = (int)blocks->size();
        const int rows = L[r] * L[r];
        for (int r0 = 0; r0 < rows; r0 += kRowsPerObsBlock)
            blocks->push_back(ObsBlock{r, r0, std::min(kRowsPerObsBlock, rows - r0)});
    }
    (*first)[nrep] = (int)blocks->size();
    return (int)blocks->size();
}

struct BLayout {
    size_t alt[3], reps, items, oblocks, first, partials, out, interval, count, status, ring, total;
};

BLayout blayout(const spin_params* p, int nrep, const int32_t* L) {
    BLayout b{};
    long long tot = 0;
    for (int r = 0; r < nrep; ++r) tot += (long long)L[r] * L[r] * L[r];
    std::vector<ObsBlock> ob;
    std::vector<int> fb;
    const int nob = obs_blocks(nrep, L, &ob, &fb);
    size_t off = 0;
    for (int c = 0; c < 3; ++c) {
        b.alt[c] = off;
        off += al(sizeof(float) * (size_t)tot);
    }
    b.reps = off;
    off += al(sizeof(BatchRep) * (size_t)nrep);
    b.items = off;
    off += al(sizeof(BatchItem) * (size_t)max_items(p, nrep, L));
    b.oblocks = off;
    off += al(sizeof(ObsBlock) * (size_t)nob);
    b.first = off;
    off += al(sizeof(int) * (size_t)(nrep + 1));
    b.partials = off;
    off += al(sizeof(double) * 5 * (size_t)nob);
    b.out = off;
    off += al(sizeof(double) * 5 * (size_t)nrep);
    b.interval = off;
    off += al(sizeof(long long));
    b.count = off;
    off += al(sizeof(long long));
    b.status = off;
    off += al(sizeof(int));
    b.ring = off;
    off += al(sizeof(double) * 5 * (size_t)nrep * SPIN_BATCH_SAMPLE_RING);
    b.total = off;
    return b;
}

StepLaunch<float> batch_launch_args(spin_batch* b, int from, bool pulse, cudaStream_t st) {
    StepLaunch<float> Ls{};
    for (int c = 0; c < 3; ++c) {
        Ls.in[c] = static_cast<const float*>(b->buf[from][c]);
        Ls.out[c] = static_cast<float*>(b->buf[from ^ 1][c]);
        Ls.hs[c] = nullptr;
    }
    Ls.g = Geom{1, 1, 1};
    Ls.ph.J = (float)b->p.J;
    Ls.ph.twoD = (float)(2.0 * b->p.D);
    for (int a = 0; a < 3; ++a) Ls.ph.H[a] = (float)b->p.H[a];
    Ls.ph.lambda = (float)b->p.lambda;
    Ls.dt = b->p.dt;
    Ls.tab = &b->tab;
    Ls.precession = b->p.precession;
    Ls.renorm = b->p.renorm;
    Ls.pulse = pulse ? 1 : 0;
    Ls.seed = b->p.seed;
    Ls.d_interval = b->d_interval;
    Ls.d_status = b->d_status;
    Ls.stream = st;
    return Ls;
}

Phys<double> bphys(const spin_batch* b) {
    Phys<double> ph{};
    ph.J = b->p.J;
    ph.twoD = 2.0 * b->p.D;
    for (int a = 0; a < 3; ++a) ph.H[a] = b->p.H[a];
    ph.lambda = b->p.lambda;
    return ph;
}

cudaError_t batch_observe(spin_batch* b, int buf, bool sample, cudaStream_t st) {
    const float* s[3] = {(const float*)b->buf[buf][0], (const float*)b->buf[buf][1], (const float*)b->buf[buf][2]};
    return launch_observables_batch(s, b->reps, b->oblocks, b->nblocks_obs, b->first_block, b->nrep, bphys(b),
                                    b->partials, b->out, sample ? b->ring : nullptr, SPIN_BATCH_SAMPLE_RING,
                                    b->d_interval, b->d_sample_count, b->p.steps_per_pulse, st);
}

// One launch per tile variant in use, each over its slice of the item table.
cudaError_t batch_step_kernels(spin_batch* b, const StepLaunch<float>& Ls) {
    for (int v = 0; v < patch_variants(); ++v) {
        const int n = b->var_first[v + 1] - b->var_first[v];
        if (n == 0) continue;
        cudaError_t e = launch_step_patch_batch(Ls, b->items + b->var_first[v], n, b->reps, v);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t batch_one_step(spin_batch* b, int from, long long n_next, cudaStream_t st) {
    const int R = b->p.steps_per_pulse;
    const bool pulse = b->p.noise && (n_next % R) == (R / 2);
    // the step kernel without its epilogue rotation, then the pulse over all
    // sites (every thread busy; same arithmetic as the single-lattice path)
    cudaError_t e = batch_step_kernels(b, batch_launch_args(b, from, false, st));
    if (e != cudaSuccess) return e;
    if (pulse) {
        float* s[3] = {(float*)b->buf[from ^ 1][0], (float*)b->buf[from ^ 1][1], (float*)b->buf[from ^ 1][2]};
        e = launch_pulse_batch(s, b->reps, b->oblocks, b->nblocks_obs, b->p.seed, b->d_interval, st);
        if (e != cudaSuccess) return e;
    }
    if (n_next % R == 0) e = batch_observe(b, from ^ 1, true, st);
    return e;
}

int class_of(const spin_batch* b, int L) {
    for (size_t c = 0; c < b->cls_L.size(); ++c)
        if (b->cls_L[c] == L) return (int)c;
    return -1;
}

void drop_graphs(spin_batch* b) {
    for (int q = 0; q < 2; ++q)
        if (b->graph[q]) {
            cudaGraphExecDestroy(b->graph[q]);
            b->graph[q] = nullptr;
        }
}

// Item and replica tables of the current class tiling, copied to the device
// (synchronous); captured graphs hold the old launch shapes and are dropped.
int upload_tables(spin_batch* b) {
    std::vector<int> var_of(b->nrep), chunk_of(b->nrep), tz;
    for (int r = 0; r < b->nrep; ++r) {
        const int c = class_of(b, b->L[r]);
        var_of[r] = b->cls_var[c];
        chunk_of[r] = b->cls_chunk[c];
    }
    b->host_items = make_items(&b->p, b->nrep, b->L.data(), var_of, chunk_of, &tz, &b->var_first);
    b->nitems = (int)b->host_items.size();
    b->host_reps.assign(b->nrep, BatchRep{});
    const double Dt = b->p.steps_per_pulse * std::fabs(b->p.dt);
    for (int r = 0; r < b->nrep; ++r) {
        b->host_reps[r].off = b->off[r];
        b->host_reps[r].L = b->L[r];
        b->host_reps[r].tz = tz[r];
        b->host_reps[r].sigma = (float)std::sqrt(2.0 * b->p.lambda * b->T[r] * Dt);
    }
    BATCH_CUDA(b, cudaStreamSynchronize(b->st));
    BATCH_CUDA(b, cudaMemcpy(b->items, b->host_items.data(), sizeof(BatchItem) * b->host_items.size(),
                             cudaMemcpyHostToDevice));
    BATCH_CUDA(b, cudaMemcpy(b->reps, b->host_reps.data(), sizeof(BatchRep) * b->host_reps.size(),
                             cudaMemcpyHostToDevice));
    drop_graphs(b);
    b->eager_intervals = 0;
    return SPIN_OK;
}

std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, int>> g_tune_cache;   // class key -> (variant, chunk)

std::string tune_key(const spin_batch* b, int L) {
    return "p" + std::to_string(b->p.precision) + "i" + std::to_string(b->p.integrator) + "L" + std::to_string(L);
}

// Device time of one step over the current tables (input buffer 0 -> buffer
// 1, no pulse, so the caller's state is untouched): the least of three.
int time_step(spin_batch* b, cudaEvent_t e0, cudaEvent_t e1, float* ms_out) {
    const StepLaunch<float> Ls = batch_launch_args(b, 0, false, b->st);
    BATCH_CUDA(b, batch_step_kernels(b, Ls));
    float ms_min = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        BATCH_CUDA(b, cudaEventRecord(e0, b->st));
        BATCH_CUDA(b, batch_step_kernels(b, Ls));
        BATCH_CUDA(b, cudaEventRecord(e1, b->st));
        BATCH_CUDA(b, cudaEventSynchronize(e1));
        float ms = 0;
        BATCH_CUDA(b, cudaEventElapsedTime(&ms, e0, e1));
        ms_min = std::min(ms_min, ms);
    }
    *ms_out = ms_min;
    return SPIN_OK;
}

// Per size class, one pass of coordinate descent on the whole batch: classes
// in decreasing order of spins, each timed over every tile variant x z-chunk
// candidate with the others held, keeping the fastest.  Pinned classes and
// classes found in the process cache are held throughout.
int autotune(spin_batch* b) {
    const int nc = (int)b->cls_L.size();
    std::vector<int> todo;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        for (int c = 0; c < nc; ++c) {
            if (b->cls_pinned[c]) continue;
            auto it = g_tune_cache.find(tune_key(b, b->cls_L[c]));
            if (it != g_tune_cache.end()) {
                b->cls_var[c] = it->second.first;
                b->cls_chunk[c] = it->second.second;
            } else {
                todo.push_back(c);
            }
        }
    }
    std::vector<long long> spins(nc, 0);
    for (int r = 0; r < b->nrep; ++r) spins[class_of(b, b->L[r])] += (long long)b->L[r] * b->L[r] * b->L[r];
    std::stable_sort(todo.begin(), todo.end(), [&](int x, int y) { return spins[x] > spins[y]; });
    cudaEvent_t e0, e1;
    BATCH_CUDA(b, cudaEventCreate(&e0));
    BATCH_CUDA(b, cudaEventCreate(&e1));
    int rc = SPIN_OK;
    for (int c : todo) {
        float best_ms = 1e30f;
        int best_v = b->cls_var[c], best_k = b->cls_chunk[c];
        for (int v = 0; v < patch_variants() && rc == SPIN_OK; ++v)
            for (int k : kChunkCandidates) {
                b->cls_var[c] = v;
                b->cls_chunk[c] = k;
                float ms = 0;
                if ((rc = upload_tables(b)) != SPIN_OK || (rc = time_step(b, e0, e1, &ms)) != SPIN_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_v = v;
                    best_k = k;
                }
            }
        b->cls_var[c] = best_v;
        b->cls_chunk[c] = best_k;
        if (rc != SPIN_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SPIN_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        for (int c : todo) g_tune_cache[tune_key(b, b->cls_L[c])] = {b->cls_var[c], b->cls_chunk[c]};
    }
    return upload_tables(b);
}

int capture_batch_interval(spin_batch* b, int from) {
    if (!b->capture_stream) BATCH_CUDA(b, cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    cudaStream_t cs = b->capture_stream;
    BATCH_CUDA(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int bb = from;
    cudaError_t e = cudaSuccess;
    for (int q = 1; q <= b->p.steps_per_pulse && e == cudaSuccess; ++q) {
        e = batch_one_step(b, bb, q, cs);
        bb ^= 1;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bset_err(b, SPIN_ECUDA, "batch interval capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaError_t e3 = cudaGraphInstantiate(&b->graph[from], g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return bset_err(b, SPIN_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e3));
    return SPIN_OK;
}

}  // namespace

extern "C" {

int spin_batch_offsets(int32_t nrep, const int32_t* L, int64_t* offsets) {
    if (nrep < 1 || !L || !offsets) return SPIN_EINVAL;
    int64_t o = 0;
    for (int r = 0; r < nrep; ++r) {
        if (L[r] < 1) return SPIN_EINVAL;
        offsets[r] = o;
        o += (int64_t)L[r] * L[r] * L[r];
    }
    offsets[nrep] = o;
    return SPIN_OK;
}

int spin_batch_workspace_size(const spin_params* p, int32_t nrep, const int32_t* L, size_t* bytes) {
    if (!bytes) return SPIN_EINVAL;
    int v = validate_batch(p, nrep, L, nullptr);
    if (v != SPIN_OK) return v;
    *bytes = blayout(p, nrep, L).total;
    return SPIN_OK;
}

int spin_batch_create(const spin_params* p, int32_t nrep, const int32_t* L, const double* T, void* sx, void* sy,
                      void* sz, int32_t chunk_planes, void* workspace, size_t workspace_bytes, void* cuda_stream,
                      spin_batch** out) {
    if (!out) return SPIN_EINVAL;
    *out = nullptr;
    int v = validate_batch(p, nrep, L, T);
    if (v != SPIN_OK) return v;
    if (!T || !sx || !sy || !sz || !workspace || reinterpret_cast<uintptr_t>(workspace) % kAlign) return SPIN_EINVAL;
    if (chunk_planes < -1) return SPIN_EINVAL;
    const BLayout Lo = blayout(p, nrep, L);
    if (workspace_bytes < Lo.total) return SPIN_ENOSPACE;
    spin_batch* b = new (std::nothrow) spin_batch();
    if (!b) return SPIN_EINVAL;
    b->p = *p;
    b->tab = tableau_for(p->integrator);
    b->nrep = nrep;
    b->L.assign(L, L + nrep);
    b->T.assign(T, T + nrep);
    b->off.resize(nrep + 1);
    spin_batch_offsets(nrep, L, b->off.data());
    b->ntot = b->off[nrep];
    b->buf[0][0] = sx;
    b->buf[0][1] = sy;
    b->buf[0][2] = sz;
    char* ws = static_cast<char*>(workspace);
    for (int c = 0; c < 3; ++c) b->buf[1][c] = ws + Lo.alt[c];
    b->st = static_cast<cudaStream_t>(cuda_stream);
    b->reps = reinterpret_cast<BatchRep*>(ws + Lo.reps);
    b->items = reinterpret_cast<BatchItem*>(ws + Lo.items);
    b->oblocks = reinterpret_cast<ObsBlock*>(ws + Lo.oblocks);
    b->first_block = reinterpret_cast<int*>(ws + Lo.first);
    b->partials = reinterpret_cast<double*>(ws + Lo.partials);
    b->out = reinterpret_cast<double*>(ws + Lo.out);
    b->d_interval = reinterpret_cast<long long*>(ws + Lo.interval);
    b->d_sample_count = reinterpret_cast<long long*>(ws + Lo.count);
    b->d_status = reinterpret_cast<int*>(ws + Lo.status);
    b->ring = reinterpret_cast<double*>(ws + Lo.ring);
    int rc = SPIN_OK;
    do {
        if (prepare_step_kernels<float>() != cudaSuccess) {
            rc = SPIN_ECUDA;
            break;
        }
        std::vector<ObsBlock> ob;
        std::vector<int> fb;
        b->nblocks_obs = obs_blocks(nrep, L, &ob, &fb);
        if (cudaMemcpy(b->oblocks, ob.data(), sizeof(ObsBlock) * ob.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b->first_block, fb.data(), sizeof(int) * fb.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemsetAsync(b->d_interval, 0, sizeof(long long), b->st) != cudaSuccess ||
            cudaMemsetAsync(b->d_sample_count, 0, sizeof(long long), b->st) != cudaSuccess ||
            cudaMemsetAsync(b->d_status, 0, sizeof(int), b->st) != cudaSuccess) {
            rc = SPIN_ECUDA;
            break;
        }
        // size classes in first-appearance order, default tiling
        for (int r = 0; r < nrep; ++r)
            if (class_of(b, L[r]) < 0) {
                b->cls_L.push_back(L[r]);
                b->cls_var.push_back(0);
                b->cls_chunk.push_back(chunk_planes > 0 ? chunk_planes : kDefaultChunk);
                b->cls_pinned.push_back(0);
            }
        rc = chunk_planes == 0 ? autotune(b) : upload_tables(b);
    } while (0);
    if (rc != SPIN_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return SPIN_OK;
}

int spin_batch_tuning(const spin_batch* b, int32_t* chunk_planes, int32_t* nitems) {
    if (!b) return SPIN_EINVAL;
    if (chunk_planes) {
        // the chunk of the class holding the most spins
        long long best = -1;
        for (size_t c = 0; c < b->cls_L.size(); ++c) {
            long long n = 0;
            for (int r = 0; r < b->nrep; ++r)
                if (b->L[r] == b->cls_L[c]) n += (long long)b->L[r] * b->L[r] * b->L[r];
            if (n > best) {
                best = n;
                *chunk_planes = b->cls_chunk[c];
            }
        }
    }
    if (nitems) *nitems = b->nitems;
    return SPIN_OK;
}

int spin_batch_tile_rows(int32_t integrator, int32_t max, int32_t* rows, int32_t* n) {
    if (!n || max < 0 || (max > 0 && !rows)) return SPIN_EINVAL;
    const Tableau tb = tableau_for(integrator);
    if (!tb.chain || !(tb.stages == 2 || tb.stages == 4)) return SPIN_EUNSUPPORTED;
    *n = patch_variants();
    for (int v = 0; v < std::min<int>(max, patch_variants()); ++v) rows[v] = patch_rows(tb.stages, v);
    return SPIN_OK;
}

int spin_batch_tiling(const spin_batch* b, int32_t max, int32_t* L, int32_t* tile_rows, int32_t* chunk, int32_t* n) {
    if (!b || !n || max < 0 || (max > 0 && (!L || !tile_rows || !chunk))) return SPIN_EINVAL;
    const int nc = (int)b->cls_L.size();
    *n = nc;
    for (int c = 0; c < std::min<int>(max, nc); ++c) {
        L[c] = b->cls_L[c];
        tile_rows[c] = patch_rows(b->tab.stages, b->cls_var[c]);
        chunk[c] = b->cls_chunk[c];
    }
    return SPIN_OK;
}

int spin_batch_set_tiling(spin_batch* b, int32_t n, const int32_t* L, const int32_t* tile_rows, const int32_t* chunk) {
    if (!b || n < 0 || (n > 0 && (!L || !tile_rows || !chunk))) return SPIN_EINVAL;
    std::vector<int> cls(n), var(n);
    for (int q = 0; q < n; ++q) {
        cls[q] = class_of(b, L[q]);
        if (cls[q] < 0) return bset_err(b, SPIN_EINVAL, "no replica has side %d", L[q]);
        var[q] = -1;
        for (int v = 0; v < patch_variants(); ++v)
            if (patch_rows(b->tab.stages, v) == tile_rows[q]) var[q] = v;
        if (var[q] < 0) return bset_err(b, SPIN_EINVAL, "tile_rows %d is not offered for this integrator", tile_rows[q]);
        if (chunk[q] < 1) return bset_err(b, SPIN_EINVAL, "chunk %d < 1", chunk[q]);
    }
    for (int q = 0; q < n; ++q) {
        b->cls_var[cls[q]] = var[q];
        b->cls_chunk[cls[q]] = chunk[q];
        b->cls_pinned[cls[q]] = 1;
    }
    return upload_tables(b);
}

int spin_batch_autotune(spin_batch* b) {
    if (!b) return SPIN_EINVAL;
    return autotune(b);
}

int spin_batch_step_pulse(spin_batch* b, int64_t nsteps) {
    if (!b || nsteps < 0) return SPIN_EINVAL;
    const int R = b->p.steps_per_pulse;
    while (nsteps > 0) {
        if (b->n % R == 0 && nsteps >= R && b->eager_intervals > 0) {
            if (!b->graph[b->cur]) {
                int rc = capture_batch_interval(b, b->cur);
                if (rc != SPIN_OK) return rc;
            }
            BATCH_CUDA(b, cudaGraphLaunch(b->graph[b->cur], b->st));
            b->n += R;
            if (R & 1) b->cur ^= 1;
            nsteps -= R;
            continue;
        }
        const bool interval_start = b->n % R == 0 && nsteps >= R;
        const int steps = interval_start ? R : 1;
        for (int q = 0; q < steps; ++q) {
            BATCH_CUDA(b, batch_one_step(b, b->cur, b->n + 1, b->st));
            b->cur ^= 1;
            b->n += 1;
        }
        nsteps -= steps;
        if (interval_start) b->eager_intervals++;
    }
    if (b->cur == 1) {
        const size_t bytes = sizeof(float) * (size_t)b->ntot;
        for (int c = 0; c < 3; ++c)
            BATCH_CUDA(b, cudaMemcpyAsync(b->buf[0][c], b->buf[1][c], bytes, cudaMemcpyDeviceToDevice, b->st));
        b->cur = 0;
    }
    return SPIN_OK;
}

int spin_batch_observables(spin_batch* b, double* out) {
    if (!b || !out) return SPIN_EINVAL;
    BATCH_CUDA(b, batch_observe(b, b->cur, false, b->st));
    int status = 0;
    BATCH_CUDA(b, cudaMemcpyAsync(out, b->out, sizeof(double) * 5 * (size_t)b->nrep, cudaMemcpyDeviceToHost, b->st));
    BATCH_CUDA(b, cudaMemcpyAsync(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    BATCH_CUDA(b, cudaStreamSynchronize(b->st));
    if (status & 1) return bset_err(b, SPIN_ETIMEOUT, "a bounded wait in the fused step gave up; the state is invalid");
    for (int r = 0; r < b->nrep; ++r)
        if (out[5 * r + 4] != 0.0) return bset_err(b, SPIN_ENONFINITE, "replica %d has non-finite spins", r);
    return SPIN_OK;
}

int spin_batch_samples(spin_batch* b, double* out, int64_t max_records, int64_t* count) {
    if (!b || !count || max_records < 0 || (max_records > 0 && !out)) return SPIN_EINVAL;
    long long total = 0;
    int status = 0;
    BATCH_CUDA(b, cudaMemcpyAsync(&total, b->d_sample_count, sizeof(total), cudaMemcpyDeviceToHost, b->st));
    BATCH_CUDA(b, cudaMemcpyAsync(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    BATCH_CUDA(b, cudaStreamSynchronize(b->st));
    if (status & 1) return bset_err(b, SPIN_ETIMEOUT, "a bounded wait in the fused step gave up; the state is invalid");
    long long first = b->samples_read;
    if (total - first > SPIN_BATCH_SAMPLE_RING) first = total - SPIN_BATCH_SAMPLE_RING;
    if (total - first > max_records) first = total - max_records;
    const long long n = total - first;
    const size_t rec = sizeof(double) * 5 * (size_t)b->nrep;
    for (long long q = 0; q < n; ++q) {
        const long long slot = (first + q) % SPIN_BATCH_SAMPLE_RING;
        BATCH_CUDA(b, cudaMemcpyAsync(out + q * 5 * b->nrep, b->ring + slot * 5 * b->nrep, rec, cudaMemcpyDeviceToHost,
                                      b->st));
    }
    BATCH_CUDA(b, cudaStreamSynchronize(b->st));
    b->samples_read = total;
    *count = n;
    return SPIN_OK;
}

int spin_batch_destroy(spin_batch* b) {
    if (!b) return SPIN_EINVAL;
    drop_graphs(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    delete b;
    return SPIN_OK;
}

const char* spin_batch_last_error(const spin_batch* b) { return b ? b->err : "null handle"; }

}  // extern "C"
