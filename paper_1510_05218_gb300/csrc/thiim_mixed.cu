// Mixed precision with FP64 defect correction (thiim_mixed_solve).
//
// The iteration x <- M x + b (one THIIM iteration, Eqs. 3-5) is run as
// iterative refinement: the FP64 defect r = (M x + b) - x of the FP64 iterate
// x is evaluated with the FP64 coefficients (the only FP64 sweep), the
// correction delta is advanced K times by the complex64 iteration
// delta <- M32 delta + r starting from delta = 0, and x += delta.  In exact
// arithmetic x + delta_K equals K plain iterations from x; with FP32
// corrections the FP64 iterate still converges to the FP64 fixed point,
// because each restart recomputes the defect in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "thiim_ctx.h"

using namespace thiim;

namespace {

struct FoldArgs {
    double2 *x[THIIM_N_FIELDS];
    const float2 *d[THIIM_N_FIELDS];
};

// x[s] += delta[s] for the 12 splits (complex128 += complex64).
__global__ void fold_kernel(const FoldArgs a, size_t n) {
    double2 *x = a.x[blockIdx.y];
    const float2 *d = a.d[blockIdx.y];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 v = x[i];
        const float2 w = d[i];
        v.x += (double)w.x;
        v.y += (double)w.y;
        x[i] = v;
    }
}

int evaluate_defect(thiim_ctx *c, void *const coeff64[THIIM_N_COEFFS], void *const x64[THIIM_N_FIELDS],
                    dim3 grid, size_t ctas, double *rel) {
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    memcpy(a.src, x64, sizeof(a.src));
    memcpy(a.dst, c->mix_r, sizeof(a.dst));
    memcpy(a.co, coeff64, sizeof(a.co));
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
    a.bc = c->bc;
    a.zchunk = c->zchunk;
    a.tiles_x = tiles_x(c);
    a.partials = c->partials;
    if (launch_defect_f64(a, grid, c->stream) != cudaSuccess) return THIIM_ERR_CUDA;
    if (finalize_norms(c->partials, ctas, c->norms, c->stream) != cudaSuccess) return THIIM_ERR_CUDA;
    double h[2];
    if (cudaMemcpyAsync(h, c->norms, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return THIIM_ERR_CUDA;
    if (!isfinite(h[0]) || !isfinite(h[1])) return THIIM_ERR_NONFINITE;
    *rel = h[1] > 0.0 ? sqrt(h[0] / h[1]) : 0.0;
    return THIIM_OK;
}

}  // namespace

extern "C" int thiim_mixed_solve(thiim_ctx *c, void *const coeff64[THIIM_N_COEFFS], void *const x64[THIIM_N_FIELDS],
                                 int inner_iters, int max_outer, double tol, int *outer_done,
                                 double *rel_residual) {
    if (!c || !coeff64 || !x64 || inner_iters < 1 || max_outer < 0) return THIIM_ERR_ARG;
    if (c->precision != THIIM_C64) return THIIM_ERR_ARG;
    if (!c->have_fields || !c->have_coeffs || c->use_table) return THIIM_ERR_STATE;
    for (int i = 0; i < THIIM_N_COEFFS; ++i) {
        if (!coeff64[i]) return THIIM_ERR_ARG;
        if (!aligned(coeff64[i], 16)) return THIIM_ERR_ALIGN;
    }
    for (int i = 0; i < THIIM_N_FIELDS; ++i) {
        if (!x64[i]) return THIIM_ERR_ARG;
        if (!aligned(x64[i], 16)) return THIIM_ERR_ALIGN;
    }
    if (!c->mix_r[0]) {
        for (int i = 0; i < THIIM_N_FIELDS; ++i) {
            if (cudaMalloc(&c->mix_r[i], c->n_cells * 8) != cudaSuccess) {
                for (int j = 0; j < i; ++j) { cudaFree(c->mix_r[j]); c->mix_r[j] = nullptr; }
                c->mix_r[i] = nullptr;
                cudaGetLastError();
                return THIIM_ERR_NOMEM;
            }
        }
    }
    const int tx = tiles_x(c), ty = tiles_y(c);
    const int chunks = (c->nz + c->zchunk - 1) / c->zchunk;
    const dim3 grid((unsigned)(tx * ty), (unsigned)chunks);
    const size_t ctas = (size_t)tx * ty * chunks;
    int st = ensure_partials(c, ctas);
    if (st) return st;
    if (!c->norms && cudaMalloc(&c->norms, 2 * sizeof(double)) != cudaSuccess) return THIIM_ERR_NOMEM;

    SweepArgs a;
    memset(&a, 0, sizeof(a));
    memcpy(a.co, c->coeff, sizeof(a.co));
    memcpy(a.xsrc, c->mix_r, sizeof(a.xsrc));
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
    a.bc = c->bc;
    a.zchunk = c->zchunk;
    a.tiles_x = tx;
    FoldArgs f;
    for (int i = 0; i < THIIM_N_FIELDS; ++i) {
        f.x[i] = (double2 *)x64[i];
        f.d[i] = (const float2 *)c->user[i];
    }
    size_t fblocks = (c->n_cells + 255) / 256;
    if (fblocks > 2048) fblocks = 2048;

    double rel = 0.0;
    int outer = 0;
    for (;; ++outer) {
        st = evaluate_defect(c, coeff64, x64, grid, ctas, &rel);
        if (st) return st;
        if (rel <= tol || outer >= max_outer) break;
        // delta <- 0, then K correction iterations delta <- M32 delta + r
        for (int i = 0; i < THIIM_N_FIELDS; ++i)
            if (cudaMemsetAsync(c->user[i], 0, c->n_cells * 8, c->stream) != cudaSuccess) return THIIM_ERR_CUDA;
        void **from = c->user, **to = c->alt;
        for (int it = 0; it < inner_iters; ++it) {
            memcpy(a.src, from, sizeof(a.src));
            memcpy(a.dst, to, sizeof(a.dst));
            if (launch_correct_f32(a, grid, c->stream) != cudaSuccess) return THIIM_ERR_CUDA;
            void **tmp = from; from = to; to = tmp;
        }
        for (int i = 0; i < THIIM_N_FIELDS; ++i) f.d[i] = (const float2 *)from[i];
        fold_kernel<<<dim3((unsigned)fblocks, THIIM_N_FIELDS), 256, 0, c->stream>>>(f, c->n_cells);
        if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
    }
    c->have_norm = false;   // the context's own fields hold a correction, not an iterate
    if (outer_done) *outer_done = outer;
    if (rel_residual) *rel_residual = rel;
    return THIIM_OK;
}
