// Magnetisation and energy per spin, accumulated in FP64 (Sec. III.A samples
// at the end of every Delta t; Sec. IV's Heisenberg energy):
//   M = (1/N) sum_i s_i
//   E = (1/N) [ -J sum_<ij> s_i.s_j - D sum_i s_iz^2 - sum_i (H + h_i).s_i ]
// each bond counted once through the three forward neighbours of every site.
// Pass 1: grid-stride FP64 partial sums, warp-shuffle then shared-memory
// reduction, one 5-double record per block.  Pass 2: one block adds the block
// records in a fixed order, so the result is bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>

#include "spin_internal.h"

namespace spin {

namespace {

constexpr int kObsThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename real, bool HSITE>
__global__ void __launch_bounds__(kObsThreads) k_obs_partial(const real* __restrict__ sx, const real* __restrict__ sy,
                                                             const real* __restrict__ sz, const real* __restrict__ hx,
                                                             const real* __restrict__ hy, const real* __restrict__ hz,
                                                             int nx, int ny, int nz, double J, double D, double H0,
                                                             double H1, double H2, double* __restrict__ partials,
                                                             int bc) {
    // one warp per lattice row (y, z); lanes stride along x, so no per-site
    // index division and the row's loads are coalesced
    const long long P = (long long)nx * ny;
    const int rows = ny * nz;
    const int lane = threadIdx.x & 31;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    double m0 = 0, m1 = 0, m2 = 0, e = 0, bad = 0;
    for (int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps_total) {
        const int y = row % ny;
        const int z = row / ny;
        const long long rb = (long long)z * P + (long long)y * nx;
        const long long rby = (long long)z * P + (long long)(y + 1 == ny ? 0 : y + 1) * nx;
        const long long rbz = (long long)(z + 1 == nz ? 0 : z + 1) * P + (long long)y * nx;
        // per-site terms in the state's precision, summed over this lane's
        // sites of the row, then added into the FP64 accumulators
        real rm0 = 0, rm1 = 0, rm2 = 0, re = 0;
        int rbad = 0;
        const real Jr = (real)J, Dr = (real)D, H0r = (real)H0, H1r = (real)H1, H2r = (real)H2;
        for (int x = lane; x < nx; x += 32) {
            const long long i = rb + x;
            const long long ix = rb + (x + 1 == nx ? 0 : x + 1);
            const long long iy = rby + x;
            const long long iz = rbz + x;
            const real a = sx[i], b = sy[i], c = sz[i];
            if (!isfinite(a) || !isfinite(b) || !isfinite(c)) rbad += 1;
            rm0 += a;
            rm1 += b;
            rm2 += c;
            // forward bonds; with free boundaries none crosses the last face
            const real wx = (bc && x + 1 == nx) ? real(0) : real(1);
            const real wy = (bc && y + 1 == ny) ? real(0) : real(1);
            const real wz = (bc && z + 1 == nz) ? real(0) : real(1);
            const real bond = a * (wx * sx[ix] + wy * sx[iy] + wz * sx[iz]) + b * (wx * sy[ix] + wy * sy[iy] + wz * sy[iz]) +
                              c * (wx * sz[ix] + wy * sz[iy] + wz * sz[iz]);
            real f0 = H0r, f1 = H1r, f2 = H2r;
            if (HSITE) {
                f0 += hx[i];
                f1 += hy[i];
                f2 += hz[i];
            }
            re += -Jr * bond - Dr * c * c - (f0 * a + f1 * b + f2 * c);
        }
        m0 += (double)rm0;
        m1 += (double)rm1;
        m2 += (double)rm2;
        e += (double)re;
        bad += (double)rbad;
    }
    __shared__ double red[kObsThreads / 32][5];
    m0 = warp_sum(m0);
    m1 = warp_sum(m1);
    m2 = warp_sum(m2);
    e = warp_sum(e);
    bad = warp_sum(bad);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[w][0] = m0;
        red[w][1] = m1;
        red[w][2] = m2;
        red[w][3] = e;
        red[w][4] = bad;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double acc = 0;
        for (int q = 0; q < kObsThreads / 32; ++q) acc += red[q][threadIdx.x];
        partials[(long long)blockIdx.x * 5 + threadIdx.x] = acc;
    }
}

__global__ void __launch_bounds__(kObsThreads) k_obs_final(const double* __restrict__ partials, int nblocks, long long N,
                                                           double* __restrict__ out5, double* __restrict__ ring, int ring_len,
                                                           long long* __restrict__ interval,
                                                           long long* __restrict__ sample_count, int R) {
    __shared__ double red[kObsThreads / 32][5];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int q = 0; q < 5; ++q) acc[q] += partials[(long long)b * 5 + q];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int q = 0; q < 5; ++q) {
        const double v = warp_sum(acc[q]);
        if (l == 0) red[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[5] = {0, 0, 0, 0, 0};
        for (int ww = 0; ww < kObsThreads / 32; ++ww)
            for (int q = 0; q < 5; ++q) t[q] += red[ww][q];
        const double invN = 1.0 / (double)N;
        out5[0] = t[0] * invN;
        out5[1] = t[1] * invN;
        out5[2] = t[2] * invN;
        out5[3] = t[3] * invN;
        out5[4] = t[4];
        if (ring) {
            const long long m = *interval;
            double* rec = ring + (*sample_count % ring_len) * 5;
            rec[0] = (double)((m + 1) * (long long)R);
            rec[1] = out5[0];
            rec[2] = out5[1];
            rec[3] = out5[2];
            rec[4] = out5[3];
            *interval = m + 1;
            *sample_count = *sample_count + 1;
        }
    }
}

// Batched replicas: the same row-wise reduction, each block on a row range
// of one replica; the final pass gives one record per replica.
__global__ void __launch_bounds__(kObsThreads) k_obs_batch_partial(const float* __restrict__ sx, const float* __restrict__ sy,
                                                                   const float* __restrict__ sz,
                                                                   const BatchRep* __restrict__ reps,
                                                                   const ObsBlock* __restrict__ blocks, double J, double D,
                                                                   double H0, double H1, double H2,
                                                                   double* __restrict__ partials) {
    const ObsBlock ob = blocks[blockIdx.x];
    const BatchRep rp = reps[ob.rep];
    const int L = rp.L;
    const long long P = (long long)L * L;
    const float* ax = sx + rp.off;
    const float* ay = sy + rp.off;
    const float* az = sz + rp.off;
    const int lane = threadIdx.x & 31;
    double m0 = 0, m1 = 0, m2 = 0, e = 0, bad = 0;
    const float Jr = (float)J, Dr = (float)D, H0r = (float)H0, H1r = (float)H1, H2r = (float)H2;
    for (int row = ob.row0 + (threadIdx.x >> 5); row < ob.row0 + ob.nrows; row += (blockDim.x >> 5)) {
        const int y = row % L, z = row / L;
        const long long rb = (long long)z * P + (long long)y * L;
        const long long rby = (long long)z * P + (long long)(y + 1 == L ? 0 : y + 1) * L;
        const long long rbz = (long long)(z + 1 == L ? 0 : z + 1) * P + (long long)y * L;
        float rm0 = 0, rm1 = 0, rm2 = 0, re = 0;
        int rbad = 0;
        for (int x = lane; x < L; x += 32) {
            const long long i = rb + x, ix = rb + (x + 1 == L ? 0 : x + 1), iy = rby + x, iz = rbz + x;
            const float a = ax[i], b = ay[i], c = az[i];
            if (!isfinite(a) || !isfinite(b) || !isfinite(c)) rbad += 1;
            rm0 += a;
            rm1 += b;
            rm2 += c;
            const float bond = a * (ax[ix] + ax[iy] + ax[iz]) + b * (ay[ix] + ay[iy] + ay[iz]) + c * (az[ix] + az[iy] + az[iz]);
            re += -Jr * bond - Dr * c * c - (H0r * a + H1r * b + H2r * c);
        }
        m0 += (double)rm0;
        m1 += (double)rm1;
        m2 += (double)rm2;
        e += (double)re;
        bad += (double)rbad;
    }
    __shared__ double red[kObsThreads / 32][5];
    m0 = warp_sum(m0);
    m1 = warp_sum(m1);
    m2 = warp_sum(m2);
    e = warp_sum(e);
    bad = warp_sum(bad);
    const int w = threadIdx.x >> 5;
    if (lane == 0) {
        red[w][0] = m0;
        red[w][1] = m1;
        red[w][2] = m2;
        red[w][3] = e;
        red[w][4] = bad;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double acc = 0;
        for (int q = 0; q < kObsThreads / 32; ++q) acc += red[q][threadIdx.x];
        partials[(long long)blockIdx.x * 5 + threadIdx.x] = acc;
    }
}

__global__ void __launch_bounds__(kObsThreads) k_obs_batch_final(const double* __restrict__ partials,
                                                                 const int* __restrict__ first_block,
                                                                 const BatchRep* __restrict__ reps, int nrep,
                                                                 double* __restrict__ out, double* __restrict__ ring,
                                                                 int ring_len, long long* __restrict__ interval,
                                                                 long long* __restrict__ sample_count, int R) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long m = ring ? *interval : 0;
    const long long slot = ring ? (*sample_count % ring_len) : 0;
    for (int r = w; r < nrep; r += blockDim.x >> 5) {
        double acc[5] = {0, 0, 0, 0, 0};
        for (int b = first_block[r] + lane; b < first_block[r + 1]; b += 32)
            for (int q = 0; q < 5; ++q) acc[q] += partials[(long long)b * 5 + q];
        for (int q = 0; q < 5; ++q) acc[q] = warp_sum(acc[q]);
        if (lane == 0) {
            const double L = (double)reps[r].L;
            const double invN = 1.0 / (L * L * L);
            double* o = out + (long long)r * 5;
            o[0] = acc[0] * invN;
            o[1] = acc[1] * invN;
            o[2] = acc[2] * invN;
            o[3] = acc[3] * invN;
            o[4] = acc[4];
            if (ring) {
                double* rec = ring + (slot * nrep + r) * 5;
                rec[0] = (double)((m + 1) * (long long)R);
                rec[1] = o[0];
                rec[2] = o[1];
                rec[3] = o[2];
                rec[4] = o[3];
            }
        }
    }
    __syncthreads();
    if (ring && threadIdx.x == 0) {
        *interval = m + 1;
        *sample_count = *sample_count + 1;
    }
}

}  // namespace

int observables_blocks(Geom g) {
    const long long rows = (long long)g.ny * g.nz;
    const long long warps_per_block = kObsThreads / 32;
    return (int)std::max<long long>(1, std::min<long long>((rows + warps_per_block - 1) / warps_per_block, 152LL * 4));
}

template <typename real>
cudaError_t launch_observables(const real* s[3], const real* hs[3], Geom g, Phys<double> ph, double* partials,
                               int nblocks, double* out5, double* sample_ring, int ring, long long* d_interval,
                               long long* d_sample_count, int R, cudaStream_t stream, int bc) {
    const double D = 0.5 * ph.twoD;
    if (hs[0])
        k_obs_partial<real, true><<<nblocks, kObsThreads, 0, stream>>>(s[0], s[1], s[2], hs[0], hs[1], hs[2], g.nx, g.ny, g.nz,
                                                                       (double)ph.J, D, (double)ph.H[0], (double)ph.H[1],
                                                                       (double)ph.H[2], partials, bc);
    else
        k_obs_partial<real, false><<<nblocks, kObsThreads, 0, stream>>>(s[0], s[1], s[2], nullptr, nullptr, nullptr, g.nx, g.ny,
                                                                        g.nz, (double)ph.J, D, (double)ph.H[0],
                                                                        (double)ph.H[1], (double)ph.H[2], partials, bc);
    k_obs_final<<<1, kObsThreads, 0, stream>>>(partials, nblocks, g.N(), out5, sample_ring, ring, d_interval,
                                               d_sample_count, R);
    return cudaGetLastError();
}

cudaError_t launch_observables_batch(const float* s[3], const BatchRep* reps, const ObsBlock* blocks, int nblocks,
                                     const int* first_block, int nrep, Phys<double> ph, double* partials,
                                     double* out, double* ring, int ring_len, long long* d_interval,
                                     long long* d_sample_count, int R, cudaStream_t stream) {
    k_obs_batch_partial<<<nblocks, kObsThreads, 0, stream>>>(s[0], s[1], s[2], reps, blocks, ph.J, 0.5 * ph.twoD,
                                                             ph.H[0], ph.H[1], ph.H[2], partials);
    k_obs_batch_final<<<1, kObsThreads, 0, stream>>>(partials, first_block, reps, nrep, out, ring, ring_len, d_interval,
                                                     d_sample_count, R);
    return cudaGetLastError();
}

template cudaError_t launch_observables<float>(const float* s[3], const float* hs[3], Geom, Phys<double>, double*, int,
                                               double*, double*, int, long long*, long long*, int, cudaStream_t, int);
template cudaError_t launch_observables<double>(const double* s[3], const double* hs[3], Geom, Phys<double>, double*,
                                                int, double*, double*, int, long long*, long long*, int, cudaStream_t,
                                                int);

}  // namespace spin

// ---------------------------------------------------------------------------
// Observables without any allocation by the library or the caller.
//
// Some callers cannot call cudaMalloc (or ask a framework to allocate) at the
// point where they want the magnetisation and energy: code running inside a
// strict memory budget, a host thread that must not take the allocator's
// lock, or a plug-in that only receives pointers to existing arrays.  For
// them this entry point keeps the reduction's scratch -- one 5-double record
// per block of the first pass -- in a fixed file-scope device array that is
// part of the loaded module, so nothing is allocated per call.
// ---------------------------------------------------------------------------

#include <mutex>

#include "../../include/spinpulse.h"

namespace spin {
namespace {

constexpr int kNoAllocMaxBlocks = SPIN_NOALLOC_MAX_BLOCKS;
// Block records of the first reduction pass, shared by every call on a device.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * 5];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so its address must come
// from cudaGetSymbolAddress, called with the device current.  Outside stream
// capture it is looked up on every call (a cudaDeviceReset reloads the module
// and may move the array); a call on a capturing stream reuses the address
// the last uncaptured call found on this device.
cudaError_t noalloc_scratch(cudaStream_t st, double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = static_cast<double*>(p);
    } else if (!g_noalloc_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace spin

extern "C" int spin_observables_noalloc(int32_t precision, const void* sx, const void* sy, const void* sz,
                                        const void* h_site, int32_t nx, int32_t ny, int32_t nz, double J, double D,
                                        const double H[3], int32_t bc, double* out5, void* cuda_stream) {
    using namespace spin;
    if (!sx || !sy || !sz || !out5 || !H) return SPIN_EINVAL;
    if (bc != 0 && bc != 1) return SPIN_EINVAL;
    if (precision != 32 && precision != 64) return SPIN_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1) return SPIN_EINVAL;
    const Geom g{nx, ny, nz};
    if (g.N() > (long long)SPIN_NOALLOC_MAX_SITES) return SPIN_EINVAL;  // beyond the stated maximum
    const int nblocks = observables_blocks(g);
    if (nblocks > kNoAllocMaxBlocks) return SPIN_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double* scratch = nullptr;
    const cudaError_t es = noalloc_scratch(st, &scratch);
    if (es == cudaErrorStreamCaptureUnsupported) return SPIN_EINVAL;
    if (es != cudaSuccess) return SPIN_ECUDA;
    Phys<double> ph{};
    ph.J = J;
    ph.twoD = 2.0 * D;
    ph.H[0] = H[0];
    ph.H[1] = H[1];
    ph.H[2] = H[2];
    const size_t comp = (size_t)(precision == 64 ? 8 : 4) * (size_t)g.N();
    cudaError_t e;
    if (precision == 32) {
        const float* s[3] = {(const float*)sx, (const float*)sy, (const float*)sz};
        const float* hs[3] = {nullptr, nullptr, nullptr};
        if (h_site)
            for (int c = 0; c < 3; ++c) hs[c] = (const float*)((const char*)h_site + c * comp);
        e = launch_observables<float>(s, hs, g, ph, scratch, nblocks, out5, nullptr, 0, nullptr, nullptr, 1, st, bc);
    } else {
        const double* s[3] = {(const double*)sx, (const double*)sy, (const double*)sz};
        const double* hs[3] = {nullptr, nullptr, nullptr};
        if (h_site)
            for (int c = 0; c < 3; ++c) hs[c] = (const double*)((const char*)h_site + c * comp);
        e = launch_observables<double>(s, hs, g, ph, scratch, nblocks, out5, nullptr, 0, nullptr, nullptr, 1, st, bc);
    }
    return e == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}
