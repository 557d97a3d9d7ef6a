// Fused FP32 step of a single lattice for chain tableaus (RK4, RK2 midpoint,
// Heun): the z-marching tile of patch_tile.cuh over the x-y tiling and z
// chunks of one lattice, the stage-storing variant the adjoint's
// recomputation uses, and the noise pulse over the finished state.
//
// Spin-plane staging: per-thread cp.async copies of each thread's column
// pair, two iterations ahead.  With SPIN_TMA=1 in the environment, RK4 on a
// lattice whose x and y sides are multiples of 4 (at least 24 and 16) with
// 16-byte aligned component arrays stages each plane by tensor-map bulk
// copies instead (TMA: nine pieces per component so that every piece lies in
// one periodic image of the lattice, one mbarrier per staging slot).  Both
// give bitwise the same results; on GB300 the TMA staging measured about
// twice the step time (27 small copies per plane and CTA against 3 cp.async
// per thread), so it is not the default.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "patch_tile.cuh"
#include "patch_tmem.cuh"

namespace spin {

namespace {

// The adjoint's recomputation runs its steps back to back as programmatic
// dependents: a store step waits for the kernel before it
// (griddepcontrol.wait; a no-op without a programmatic dependency) before it
// touches global memory, and lets the next launch once all of its CTAs are
// done, so a launch overlaps the drain of its predecessor.  (The plain steps,
// replayed in whole-interval graphs, measured no gain from it: 0.530 against
// 0.527 ms per 128^3 interval.)
__device__ __forceinline__ void dependent_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void dependents_go() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
template <typename Kern, typename... Args>
cudaError_t launch_dependent(Kern kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int S, bool PREC, bool HSITE, bool PULSE>
__global__ void __launch_bounds__(kPT* PatchShape<S>::TY, 1) k_step_patch(PatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    patch_tile<S, PREC, HSITE, PULSE, false, 0>(a, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                                             reinterpret_cast<float*>(smem_raw));
}

// The same step that also writes every stage's input and increment at the
// output sites (the adjoint reads them instead of recomputing the stages).
template <int S, bool PREC, bool HSITE>
__global__ void __launch_bounds__(kPT* PatchShape<S>::TY, 1) k_step_patch_store(PatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dependent_wait();
    patch_tile<S, PREC, HSITE, false, true, 0>(a, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
                                            reinterpret_cast<float*>(smem_raw));
    dependents_go();
}

// RK4 step with the spin planes staged by TMA; the tensor maps live in the
// kernel's parameter space.
template <int S, bool PREC, bool HSITE, bool STORE>
__global__ void __launch_bounds__(kPT* PatchShape<S>::TY, 1)
    k_step_patch_tma(PatchArgs a, const __grid_constant__ TmaMaps maps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // pieces are copied to 128-byte boundaries of the staging ring
    float* sh = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    patch_tile<S, PREC, HSITE, false, STORE, 0, true>(a, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, sh,
                                                      &maps);
}

// RK4 step with the spin and accumulator rings of its older planes in tensor
// memory and 28-row tiles (patch_tmem.cuh).
template <bool PREC>
__global__ void __launch_bounds__(kPT* PatchShape<4, kTmemVariant>::TY, 1) k_step_patch_tmem(PatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned tm_slot;
    tm_tile<PREC>(a, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, reinterpret_cast<float*>(smem_raw), &tm_slot);
}

template <bool PREC>
cudaError_t patch_tmem_launch(const PatchArgs& a, dim3 grid, cudaStream_t st, bool prepare) {
    const size_t smem = patch_smem<4, PREC, false, false, kTmemVariant>();
    if (prepare)
        return cudaFuncSetAttribute(k_step_patch_tmem<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_step_patch_tmem<PREC><<<grid, dim3(kPT, PatchShape<4, kTmemVariant>::TY), smem, st>>>(a);
    return cudaGetLastError();
}

// z chunks of a tiling: one resident CTA per SM, so the chunk length that
// minimises waves x (chunk planes + pipeline fill of 2S-2 iterations); the
// returned cost is that product
int choose_chunk(int nz, long long tiles, int S, double* cost) {
    int best_chunks = 1;
    double best_cost = 1e300;
    for (int c = 1; c <= std::max(1, nz / 4); ++c) {
        const int zc_c = (nz + c - 1) / c;
        const int used = (nz + zc_c - 1) / zc_c;
        const long long ctas = tiles * used;
        const double waves = (double)((ctas + 151) / 152);
        const double cst = waves * (zc_c + 2 * S - 2);
        if (cst < best_cost - 1e-9) {
            best_cost = cst;
            best_chunks = c;
        }
    }
    if (cost) *cost = best_cost;
    return (nz + best_chunks - 1) / best_chunks;
}

template <int S>
size_t patch_tma_smem() {
    constexpr int ROWS = PatchShape<S>::PY * PatchShape<S>::TY;
    return sizeof(float) * (2 * S * 3 * ROWS * kRS + 4 * TmaSlot<ROWS>::SLOT) + 4 * sizeof(unsigned long long) + 128;
}

template <int S, bool PREC, bool HSITE, bool PULSE>
cudaError_t patch_launch(const PatchArgs& a, dim3 grid, cudaStream_t st, bool prepare) {
    const size_t smem = patch_smem<S, PREC, HSITE, PULSE>();
    if (prepare)
        return cudaFuncSetAttribute(k_step_patch<S, PREC, HSITE, PULSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    k_step_patch<S, PREC, HSITE, PULSE><<<grid, dim3(kPT, PatchShape<S>::TY), smem, st>>>(a);
    return cudaGetLastError();
}

template <int S, bool PREC, bool HSITE>
cudaError_t patch_store_launch(const PatchArgs& a, dim3 grid, cudaStream_t st, bool prepare) {
    const size_t smem = patch_smem<S, PREC, HSITE, false>();
    if (prepare)
        return cudaFuncSetAttribute(k_step_patch_store<S, PREC, HSITE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    return launch_dependent(k_step_patch_store<S, PREC, HSITE>, grid, dim3(kPT, PatchShape<S>::TY), smem, st, a);
}

template <int S, bool PREC, bool HSITE, bool STORE>
cudaError_t patch_tma_launch(const PatchArgs& a, const TmaMaps* maps, dim3 grid, cudaStream_t st, bool prepare) {
    const size_t smem = patch_tma_smem<S>();
    if (prepare)
        return cudaFuncSetAttribute(k_step_patch_tma<S, PREC, HSITE, STORE>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_step_patch_tma<S, PREC, HSITE, STORE><<<grid, dim3(kPT, PatchShape<S>::TY), smem, st>>>(a, *maps);
    return cudaGetLastError();
}

template <int S>
cudaError_t patch_tma_dispatch(const PatchArgs& a, const TmaMaps* maps, dim3 grid, cudaStream_t st, bool prec,
                               bool hs, bool store, bool prepare) {
#define SPIN_TMA_CASE(P_, H_, T_)                                                       \
    if (prepare) {                                                                      \
        cudaError_t e = patch_tma_launch<S, P_, H_, T_>(a, maps, grid, st, true);       \
        if (e != cudaSuccess) return e;                                                 \
    } else if (prec == P_ && hs == H_ && store == T_) {                                 \
        return patch_tma_launch<S, P_, H_, T_>(a, maps, grid, st, false);               \
    }
    SPIN_TMA_CASE(true, false, false)
    SPIN_TMA_CASE(true, true, false)
    SPIN_TMA_CASE(false, false, false)
    SPIN_TMA_CASE(false, true, false)
#undef SPIN_TMA_CASE
    return prepare ? cudaSuccess : cudaErrorInvalidValue;
}

template <int S>
cudaError_t patch_store_dispatch(const PatchArgs& a, dim3 grid, cudaStream_t st, bool prec, bool hs, bool prepare) {
    if (prepare) {
        cudaError_t e;
        if ((e = patch_store_launch<S, true, false>(a, grid, st, true)) != cudaSuccess) return e;
        if ((e = patch_store_launch<S, true, true>(a, grid, st, true)) != cudaSuccess) return e;
        if ((e = patch_store_launch<S, false, false>(a, grid, st, true)) != cudaSuccess) return e;
        return patch_store_launch<S, false, true>(a, grid, st, true);
    }
    if (prec) return hs ? patch_store_launch<S, true, true>(a, grid, st, false)
                        : patch_store_launch<S, true, false>(a, grid, st, false);
    return hs ? patch_store_launch<S, false, true>(a, grid, st, false) : patch_store_launch<S, false, false>(a, grid, st, false);
}

template <int S>
cudaError_t patch_dispatch(const PatchArgs& a, dim3 grid, cudaStream_t st, bool prec, bool hs, bool pulse,
                           bool prepare) {
#define SPIN_PATCH_CASE(P_, H_, U_)                                                   \
    if (prepare) {                                                                    \
        cudaError_t e = patch_launch<S, P_, H_, U_>(a, grid, st, true);               \
        if (e != cudaSuccess) return e;                                               \
    } else if (prec == P_ && hs == H_ && pulse == U_) {                               \
        return patch_launch<S, P_, H_, U_>(a, grid, st, false);                       \
    }
    SPIN_PATCH_CASE(true, false, false)
    SPIN_PATCH_CASE(true, true, false)
    SPIN_PATCH_CASE(false, false, false)
    SPIN_PATCH_CASE(false, true, false)
#undef SPIN_PATCH_CASE
    return prepare ? cudaSuccess : cudaErrorInvalidValue;
}

// The noise pulse on its own, over every site of the lattice (all threads
// busy): on pulse steps of a single lattice the step kernel runs without its
// epilogue rotation and this kernel rotates the finished state in place.  The
// arithmetic per site is the fused epilogue's, so the results are identical.
__global__ void __launch_bounds__(256) k_pulse_f32(float* __restrict__ sx, float* __restrict__ sy, float* __restrict__ sz,
                                                   long long N, uint64_t seed, const long long* __restrict__ interval,
                                                   uint64_t replica, float sigma) {
    const uint64_t k = (uint64_t)*interval;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float x = sx[i], y = sy[i], z = sz[i];
        pulse_site<float>(x, y, z, seed, (uint64_t)i, k, replica, sigma);
        sx[i] = x;
        sy[i] = y;
        sz[i] = z;
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if the driver does not provide it
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// TMA staging is selected by SPIN_TMA=1 and applies to RK4 on a lattice whose
// x side is a multiple of 4 and at least 24, whose y side is a multiple of 4
// and at least the tile's output height, with 16-byte aligned component
// arrays (every tensor-map stride is then a multiple of 16 bytes).
bool tma_applies(const PatchArgs& a, int S) {
    if (S != 4) return false;
    const char* env = std::getenv("SPIN_TMA");
    if (!env || env[0] != '1') return false;
    const int outy = PatchShape<4>::PY * PatchShape<4>::TY - 8;
    const uintptr_t al = reinterpret_cast<uintptr_t>(a.in0) | reinterpret_cast<uintptr_t>(a.in1) |
                         reinterpret_cast<uintptr_t>(a.in2);
    return (a.nx % 4) == 0 && (a.ny % 4) == 0 && a.nx >= 24 && a.ny >= outy && (al & 15) == 0 &&
           tensor_map_encoder() != nullptr;
}

// Per component, one map per piece shape: (4 | 24 columns) x (4 | ROWS-8 rows)
// x 1 plane over the (nx, ny, nz) array; out-of-range boxes never occur (each
// piece is copied at its wrapped origin).
bool encode_tma_maps(const PatchArgs& a, TmaMaps* maps) {
    constexpr int ROWS = PatchShape<4>::PY * PatchShape<4>::TY;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    const float* comp[3] = {a.in0, a.in1, a.in2};
    const cuuint64_t dims[3] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)a.nx * 4, (cuuint64_t)a.nx * (cuuint64_t)a.ny * 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int c = 0; c < 3; ++c)
        for (int shape = 0; shape < 4; ++shape) {
            const cuuint32_t box[3] = {(cuuint32_t)((shape & 1) ? 24 : 4), (cuuint32_t)((shape & 2) ? ROWS - 8 : 4), 1};
            const CUresult r = enc(&maps->m[c][shape], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                                   const_cast<float*>(comp[c]), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return false;
        }
    return true;
}

}  // namespace

cudaError_t prepare_patch_batch_kernels();

cudaError_t prepare_patch_kernels() {
    cudaError_t e = prepare_patch_batch_kernels();
    if (e != cudaSuccess) return e;
    PatchArgs a{};
    e = patch_dispatch<4>(a, dim3(1), 0, false, false, false, true);
    if (e != cudaSuccess) return e;
    e = patch_dispatch<2>(a, dim3(1), 0, false, false, false, true);
    if (e != cudaSuccess) return e;
    e = patch_store_dispatch<4>(a, dim3(1), 0, false, false, true);
    if (e != cudaSuccess) return e;
    e = patch_store_dispatch<2>(a, dim3(1), 0, false, false, true);
    if (e != cudaSuccess) return e;
    if ((e = patch_tmem_launch<true>(a, dim3(1), 0, true)) != cudaSuccess) return e;
    if ((e = patch_tmem_launch<false>(a, dim3(1), 0, true)) != cudaSuccess) return e;
    return patch_tma_dispatch<4>(a, nullptr, dim3(1), 0, false, false, false, true);
}

cudaError_t launch_step_patch(const StepLaunch<float>& L) {
    const int S = L.tab->stages;
    PatchArgs a = patch_args_common(L);
    const bool hs = L.hs[0] != nullptr;
    const bool store = L.st_n[0][0] != nullptr;
    const int outx = kPC - 2 * S;
    const int tiles_x = (L.g.nx + outx - 1) / outx;
    // register-ring tiling (24 rows for RK4) ...
    const int outy = patch_out_y(S, 0);
    const int tiles_y = (L.g.ny + outy - 1) / outy;
    double cost = 0;
    int zc = choose_chunk(L.g.nz, (long long)tiles_x * tiles_y, S, &cost);
    dim3 grid(tiles_x, tiles_y, (L.g.nz + zc - 1) / zc);
    // ... or, for a plain RK4 step staged by cp.async, the TMEM-ring tiling
    // (28 rows) where its estimated time, waves x iterations x tile rows, is
    // lower (SPIN_TMEM=0 / =1 in the environment forbids / forces it)
    const bool use_tma = !store && tma_applies(a, S);
    bool tmem = false;
    if (S == 4 && !hs && !store && !use_tma) {
        const char* env = std::getenv("SPIN_TMEM");
        if (!env || env[0] != '0') {
            constexpr int rows_r = PatchShape<4, 0>::TY, rows_t = PatchShape<4, kTmemVariant>::TY;
            const int ty_t = (L.g.ny + (rows_t - 8) - 1) / (rows_t - 8);
            double cost_t = 0;
            const int zc_t = choose_chunk(L.g.nz, (long long)tiles_x * ty_t, S, &cost_t);
            if ((env && env[0] == '1') || cost_t * rows_t < cost * rows_r) {
                tmem = true;
                zc = zc_t;
                grid = dim3(tiles_x, ty_t, (L.g.nz + zc_t - 1) / zc_t);
            }
        }
    }
    a.tz = zc;
    a.n_iter = zc + 2 * S - 2;
    const bool prec = L.precession != 0;
    cudaError_t e;
    if (store) {
        for (int c = 0; c < 3; ++c) {
            for (int j = 0; j < S; ++j) {
                a.stn[j][c] = L.st_n[j][c];
                if (j + 1 < S) a.stx[j][c] = L.st_x[j][c];
            }
            a.sty[c] = L.st_y[c];
        }
        a.dt = (float)L.dt;
    }
    TmaMaps maps;
    if (tmem) {
        e = prec ? patch_tmem_launch<true>(a, grid, L.stream, false) : patch_tmem_launch<false>(a, grid, L.stream, false);
    } else if (use_tma && encode_tma_maps(a, &maps)) {
        e = patch_tma_dispatch<4>(a, &maps, grid, L.stream, prec, hs, store, false);
    } else if (store) {
        e = S == 4 ? patch_store_dispatch<4>(a, grid, L.stream, prec, hs, false)
                   : patch_store_dispatch<2>(a, grid, L.stream, prec, hs, false);
    } else {
        e = S == 4 ? patch_dispatch<4>(a, grid, L.stream, prec, hs, false, false)
                   : patch_dispatch<2>(a, grid, L.stream, prec, hs, false, false);
    }
    if (e != cudaSuccess || !L.pulse) return e;
    return launch_pulse_lattice(L);
}

cudaError_t launch_pulse_lattice(const StepLaunch<float>& L) {
    const long long N = L.g.N();
    const int blocks = (int)std::max<long long>(1, std::min<long long>((N + 255) / 256, 152LL * 8));
    k_pulse_f32<<<blocks, 256, 0, L.stream>>>(L.out[0], L.out[1], L.out[2], N, L.seed, L.d_interval, L.replica,
                                              L.sigma);
    return cudaGetLastError();
}

}  // namespace spin
