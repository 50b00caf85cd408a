// thiim_step_noalloc: one sweep iteration that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator hooks, processes whose device memory
// is fully reserved up front, and hosts that only hand out pre-registered
// buffers.  For them this entry point runs one THIIM iteration from caller
// buffers to caller buffers and keeps its only scratch — the per-CTA partial
// norms of the residual reduction — in a fixed file-scope device array
// instead of an allocation.  The library has no counterpart of this in the
// paper; it is a deployment convenience.
//
// The array lives in every GPU that loads the library until the process
// exits (NOALLOC_MAX_CTAS * 16 bytes + 16 bytes = 256 KiB + 16 B).  All calls
// share it, so calls whose work overlaps on the GPU (different streams, or
// different host threads on the same device) race on it.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "../../include/thiim.h"
#include "thiim_internal.h"

using namespace thiim;

namespace {

// Largest number of sweep CTAs one call may use; bigger grids are rejected.
constexpr size_t NOALLOC_MAX_CTAS = 16384;

// partials[2*i], partials[2*i+1] for CTA i, then the two final norms.
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_CTAS + 2];

// Device address of the array on the current device.  The name
// g_noalloc_scratch in host code is only a host-side handle; kernels must be
// given the address cudaGetSymbolAddress returns.  It is looked up on every
// call that needs it (a host-side table lookup once the library's device code
// is loaded), so a context that was reset and reloaded the module never sees
// a stale address.  The first lookup on a device loads that code.
int scratch_for_current_device(double **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return THIIM_ERR_CUDA;
    }
    *out = (double *)p;
    return THIIM_OK;
}

// Sum the CTA partials in a fixed order into the last two slots.  Device
// code names the array directly.
__global__ void noalloc_finalize(size_t n) {
    __shared__ double sd[256], sx[256];
    double d = 0.0, x = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        d += g_noalloc_scratch[2 * i];
        x += g_noalloc_scratch[2 * i + 1];
    }
    sd[threadIdx.x] = d;
    sx[threadIdx.x] = x;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sd[threadIdx.x] += sd[threadIdx.x + o];
            sx[threadIdx.x] += sx[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        g_noalloc_scratch[2 * NOALLOC_MAX_CTAS] = sd[0];
        g_noalloc_scratch[2 * NOALLOC_MAX_CTAS + 1] = sx[0];
    }
}

bool aligned_to(const void *p, size_t a) { return ((size_t)p % a) == 0; }

}  // namespace

namespace thiim {

// The FP64 sweep on 32 x 8 tiles (this entry point's tiling for both
// precisions; thiim_iterate's FP64 tile is 32 x 16).
cudaError_t launch_sweep_f64_t8(const SweepArgs &a, dim3 grid, cudaStream_t s) {
    sweep_kernel<Native<double>, SWEEP_TX, SWEEP_TY, SWEEP_NT, SWEEP_MINB><<<grid, SWEEP_NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace thiim

extern "C" int thiim_step_noalloc(int nx, int ny, int nz, int precision, unsigned bc_flags,
                                  void *const src[THIIM_N_FIELDS], void *const dst[THIIM_N_FIELDS],
                                  void *const coeff[THIIM_N_COEFFS], void *cuda_stream,
                                  double *rel_residual) {
    if (nx < 1 || ny < 1 || nz < 1 || !src || !dst || !coeff) return THIIM_ERR_ARG;
    if (precision != THIIM_C128 && precision != THIIM_C64) return THIIM_ERR_ARG;
    if (bc_flags & ~7u) return THIIM_ERR_ARG;
    if ((double)nx * ny * nz > (double)(1ull << 40)) return THIIM_ERR_ARG;
    const size_t elem = precision == THIIM_C128 ? 16 : 8;
    for (int i = 0; i < THIIM_N_FIELDS; ++i) {
        if (!src[i] || !dst[i]) return THIIM_ERR_ARG;
        if (!aligned_to(src[i], elem) || !aligned_to(dst[i], elem)) return THIIM_ERR_ALIGN;
        if (src[i] == dst[i]) return THIIM_ERR_ARG;   // the sweep reads and writes different sets
    }
    for (int i = 0; i < THIIM_N_COEFFS; ++i) {
        if (!coeff[i]) return THIIM_ERR_ARG;
        if (!aligned_to(coeff[i], elem)) return THIIM_ERR_ALIGN;
    }
    // Same tiling as thiim_iterate, with the z chunking capped so the grid
    // fits the fixed partials array.
    const long tx = (nx + SWEEP_TX - 1) / SWEEP_TX, ty = (ny + SWEEP_TY - 1) / SWEEP_TY;
    const long tiles = tx * ty;
    if ((size_t)tiles > NOALLOC_MAX_CTAS) return THIIM_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return THIIM_ERR_CUDA;
    long chunks = (8L * nsm + tiles - 1) / tiles;
    const long maxchunks = nz / 8 > 0 ? nz / 8 : 1;
    if (chunks > maxchunks) chunks = maxchunks;
    if (chunks > (long)(NOALLOC_MAX_CTAS / tiles)) chunks = (long)(NOALLOC_MAX_CTAS / tiles);
    if (chunks < 1) chunks = 1;
    const int zchunk = (int)((nz + chunks - 1) / chunks);
    chunks = (nz + zchunk - 1) / zchunk;
    const size_t ctas = (size_t)tiles * chunks;

    double *scratch = nullptr;
    if (rel_residual) {
        const int st = scratch_for_current_device(&scratch);
        if (st) return st;
    }
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    memcpy(a.src, src, sizeof(a.src));
    memcpy(a.dst, dst, sizeof(a.dst));
    memcpy(a.co, coeff, sizeof(a.co));
    a.nx = nx; a.ny = ny; a.nz = nz;
    a.bc = bc_flags;
    a.zchunk = zchunk;
    a.tiles_x = (int)tx;
    a.partials = scratch;   // nullptr: no reduction
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const dim3 grid((unsigned)tiles, (unsigned)chunks);
    cudaError_t e = precision == THIIM_C128 ? launch_sweep_f64_t8(a, grid, s) : launch_sweep_f32(a, grid, s);
    if (e != cudaSuccess) return THIIM_ERR_CUDA;
    if (!rel_residual) return THIIM_OK;
    noalloc_finalize<<<1, 256, 0, s>>>(ctas);
    if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
    double h[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(h, scratch + 2 * NOALLOC_MAX_CTAS, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return THIIM_ERR_CUDA;
    if (!isfinite(h[0]) || !isfinite(h[1])) return THIIM_ERR_NONFINITE;
    *rel_residual = h[1] > 0.0 ? sqrt(h[0] / h[1]) : 0.0;
    return THIIM_OK;
}
