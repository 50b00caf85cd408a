// Absorbed power of the current iterate: P = 1/2 sum_cells sigma |E|^2, the
// quantity whose ratio to the incident power is a solar cell's absorption at
// one wavelength and polarisation.  See include/thiim.h.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/thiim.h"
#include "thiim_ctx.h"

using namespace thiim;

namespace {

constexpr int POWER_THREADS = 256;

struct PowerArgs {
    const void *e[6];        // Exy Exz Eyx Eyz Ezx Ezy
    const double *sigma;
    size_t n;
    double *partials;        // 2 per CTA: (sum, 0), summed by finalize_norms
};

template <typename V>
__device__ __forceinline__ double2 ld(const void *b, size_t i) {
    const V v = reinterpret_cast<const V *>(b)[i];
    return make_double2((double)v.x, (double)v.y);
}

// Each CTA sums a fixed grid-stride share in FP64 and reduces it in a fixed
// order; the per-CTA sums are added in a fixed order afterwards, so the result
// does not depend on scheduling.
template <typename V>
__global__ void __launch_bounds__(POWER_THREADS) power_kernel(const PowerArgs a) {
    __shared__ double red[POWER_THREADS / 32];
    double acc = 0.0;
    for (size_t p = (size_t)blockIdx.x * POWER_THREADS + threadIdx.x; p < a.n; p += (size_t)gridDim.x * POWER_THREADS) {
        const double s = a.sigma[p];
        if (s != 0.0) {
            double e2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double2 u = ld<V>(a.e[2 * c], p), w = ld<V>(a.e[2 * c + 1], p);
                const double re = u.x + w.x, im = u.y + w.y;
                e2 += re * re + im * im;
            }
            acc += s * e2;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < POWER_THREADS / 32; ++i) t += red[i];
        a.partials[2 * blockIdx.x] = 0.5 * t;
        a.partials[2 * blockIdx.x + 1] = 0.0;
    }
}

}  // namespace

extern "C" int thiim_absorbed_power(thiim_ctx *c, const double *sigma, double *power) {
    if (!c || !sigma || !power) return THIIM_ERR_ARG;
    if (!aligned(sigma, 8)) return THIIM_ERR_ALIGN;
    if (!c->have_fields) return THIIM_ERR_STATE;
    const size_t ctas = 4 * (size_t)c->num_sms;
    int st = ensure_partials(c, ctas);
    if (st) return st;
    if (!c->power && cudaMalloc(&c->power, 2 * sizeof(double)) != cudaSuccess) return THIIM_ERR_NOMEM;
    PowerArgs a;
    for (int i = 0; i < 6; ++i) a.e[i] = c->user[6 + i];
    a.sigma = sigma;
    a.n = c->n_cells;
    a.partials = c->partials;
    if (c->precision == THIIM_C64)
        power_kernel<float2><<<(unsigned)ctas, POWER_THREADS, 0, c->stream>>>(a);
    else
        power_kernel<double2><<<(unsigned)ctas, POWER_THREADS, 0, c->stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
    if (finalize_norms(c->partials, ctas, c->power, c->stream) != cudaSuccess) return THIIM_ERR_CUDA;
    double h[2];
    if (cudaMemcpyAsync(h, c->power, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return THIIM_ERR_CUDA;
    if (!isfinite(h[0])) return THIIM_ERR_NONFINITE;
    *power = h[0];
    return THIIM_OK;
}
