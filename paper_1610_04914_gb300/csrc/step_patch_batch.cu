// Batched replicas of the fused FP32 step: one CTA per work item (replica,
// x tile, y tile, z chunk) with the tile variant chosen per replica size,
// the batched noise pulse, and the tile-geometry queries the batch planner
// uses.  The tile itself is the single-lattice kernels' (patch_tile.cuh).
#include <cuda_runtime.h>

#include "patch_tile.cuh"

namespace spin {

namespace {

// Batched replicas: one CTA per work item (replica, x tile, y tile, z chunk)
// of a table sorted by cost; each replica is a cubic periodic lattice of side
// L at its own offset in the concatenated arrays, with its own pulse angle
// scale (temperature) and its index as the noise counter's replica word.
template <int S, bool PREC, bool PULSE, int V>
__global__ void __launch_bounds__(kPT* PatchShape<S, V>::TY, 1)
    k_step_patch_batch(PatchArgs base, const BatchItem* __restrict__ items, const BatchRep* __restrict__ reps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchItem it = items[blockIdx.x];
    const BatchRep rp = reps[it.rep];
    PatchArgs a = base;
    a.in0 += rp.off;
    a.in1 += rp.off;
    a.in2 += rp.off;
    a.out0 += rp.off;
    a.out1 += rp.off;
    a.out2 += rp.off;
    a.nx = a.ny = a.nz = rp.L;
    a.pair8 = pairs_aligned(rp.L, a.in0, a.in1, a.in2) ? 1 : 0;
    a.pair8out = pairs_aligned(rp.L, a.out0, a.out1, a.out2) ? 1 : 0;
    a.tz = rp.tz;
    a.n_iter = rp.tz + 2 * S - 2;
    a.sigma = rp.sigma;
    a.replica = (uint64_t)it.rep;
    patch_tile<S, PREC, false, PULSE, false, V>(a, it.bx, it.by, it.bz, reinterpret_cast<float*>(smem_raw));
}

template <int S, bool PREC, bool PULSE, int V>
cudaError_t batch_launch(const PatchArgs& a, const BatchItem* items, int nitems, const BatchRep* reps, cudaStream_t st,
                         bool prepare) {
    const size_t smem = patch_smem<S, PREC, false, PULSE, V>();
    if (prepare)
        return cudaFuncSetAttribute(k_step_patch_batch<S, PREC, PULSE, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    if (nitems <= 0) return cudaSuccess;
    k_step_patch_batch<S, PREC, PULSE, V><<<nitems, dim3(kPT, PatchShape<S, V>::TY), smem, st>>>(a, items, reps);
    return cudaGetLastError();
}

template <int S, int V>
cudaError_t batch_dispatch_v(const PatchArgs& a, const BatchItem* items, int nitems, const BatchRep* reps,
                             cudaStream_t st, bool prec, bool pulse, bool prepare) {
    if (prepare) {
        cudaError_t e;
        if ((e = batch_launch<S, true, false, V>(a, items, nitems, reps, st, true)) != cudaSuccess) return e;
        if ((e = batch_launch<S, true, true, V>(a, items, nitems, reps, st, true)) != cudaSuccess) return e;
        if ((e = batch_launch<S, false, false, V>(a, items, nitems, reps, st, true)) != cudaSuccess) return e;
        return batch_launch<S, false, true, V>(a, items, nitems, reps, st, true);
    }
    if (prec) return pulse ? batch_launch<S, true, true, V>(a, items, nitems, reps, st, false)
                           : batch_launch<S, true, false, V>(a, items, nitems, reps, st, false);
    return pulse ? batch_launch<S, false, true, V>(a, items, nitems, reps, st, false)
                 : batch_launch<S, false, false, V>(a, items, nitems, reps, st, false);
}

template <int S>
cudaError_t batch_dispatch(const PatchArgs& a, const BatchItem* items, int nitems, const BatchRep* reps,
                           cudaStream_t st, bool prec, bool pulse, bool prepare, int variant) {
    if (prepare) {
        cudaError_t e;
        if ((e = batch_dispatch_v<S, 0>(a, items, nitems, reps, st, prec, pulse, true)) != cudaSuccess) return e;
        if ((e = batch_dispatch_v<S, 1>(a, items, nitems, reps, st, prec, pulse, true)) != cudaSuccess) return e;
        return batch_dispatch_v<S, 2>(a, items, nitems, reps, st, prec, pulse, true);
    }
    switch (variant) {
        case 0: return batch_dispatch_v<S, 0>(a, items, nitems, reps, st, prec, pulse, false);
        case 1: return batch_dispatch_v<S, 1>(a, items, nitems, reps, st, prec, pulse, false);
        case 2: return batch_dispatch_v<S, 2>(a, items, nitems, reps, st, prec, pulse, false);
        default: return cudaErrorInvalidValue;
    }
}
// Batched pulse: block b rotates the sites of rows [row0, row0+nrows) of
// replica rep (the observables' block table), with that replica's angle scale
// and noise stream; same per-site arithmetic as the single-lattice kernel.
__global__ void __launch_bounds__(256) k_pulse_batch(float* __restrict__ sx, float* __restrict__ sy,
                                                     float* __restrict__ sz, const BatchRep* __restrict__ reps,
                                                     const ObsBlock* __restrict__ blocks, uint64_t seed,
                                                     const long long* __restrict__ interval) {
    const ObsBlock ob = blocks[blockIdx.x];
    const BatchRep rp = reps[ob.rep];
    const uint64_t k = (uint64_t)*interval;
    const long long first = (long long)ob.row0 * rp.L;
    const long long count = (long long)ob.nrows * rp.L;
    for (long long q = threadIdx.x; q < count; q += blockDim.x) {
        const long long i = first + q;          // site index within the replica
        const long long g = rp.off + i;
        float x = sx[g], y = sy[g], z = sz[g];
        pulse_site<float>(x, y, z, seed, (uint64_t)i, k, (uint64_t)ob.rep, rp.sigma);
        sx[g] = x;
        sy[g] = y;
        sz[g] = z;
    }
}


}  // namespace

cudaError_t launch_pulse_batch(float* s[3], const BatchRep* reps, const ObsBlock* blocks, int nblocks, uint64_t seed,
                               const long long* d_interval, cudaStream_t st) {
    k_pulse_batch<<<nblocks, 256, 0, st>>>(s[0], s[1], s[2], reps, blocks, seed, d_interval);
    return cudaGetLastError();
}
int patch_out_x(int stages) { return kPC - 2 * stages; }
int patch_rows(int stages, int variant) {
    if (stages == 4)
        return variant == 1 ? PatchShape<4, 1>::TY : (variant == 2 ? PatchShape<4, 2>::TY : PatchShape<4, 0>::TY);
    return PatchShape<2, 0>::PY *
           (variant == 1 ? PatchShape<2, 1>::TY : (variant == 2 ? PatchShape<2, 2>::TY : PatchShape<2, 0>::TY));
}
int patch_out_y(int stages, int variant) { return patch_rows(stages, variant) - 2 * stages; }
int patch_variants() { return kTileVariants; }

cudaError_t launch_step_patch_batch(const StepLaunch<float>& L, const BatchItem* items, int nitems,
                                    const BatchRep* reps, int variant) {
    const PatchArgs a = patch_args_common(L);
    const bool prec = L.precession != 0;
    if (L.tab->stages == 4)
        return batch_dispatch<4>(a, items, nitems, reps, L.stream, prec, L.pulse != 0, false, variant);
    return batch_dispatch<2>(a, items, nitems, reps, L.stream, prec, L.pulse != 0, false, variant);
}


// dynamic shared-memory limits of every batched instantiation
cudaError_t prepare_patch_batch_kernels() {
    PatchArgs a{};
    cudaError_t e = batch_dispatch<4>(a, nullptr, 0, nullptr, 0, false, false, true, 0);
    if (e != cudaSuccess) return e;
    return batch_dispatch<2>(a, nullptr, 0, nullptr, 0, false, false, true, 0);
}

}  // namespace spin
