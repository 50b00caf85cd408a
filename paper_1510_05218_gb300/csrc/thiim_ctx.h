// The library context and helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/thiim.h"
#include "thiim_internal.h"

struct thiim_ctx {
    int nx, ny, nz;
    int precision;
    unsigned bc;
    cudaStream_t stream;
    int device;
    int num_sms;
    size_t elem;                 // bytes per complex element
    size_t n_cells;
    void *coeff[THIIM_N_COEFFS];
    void *user[THIIM_N_FIELDS];  // caller's field arrays (hold x^n between calls)
    void *alt[THIIM_N_FIELDS];   // library's second field set
    void *pair_co[THIIM_N_COEFFS];  // THIIM_C128_PAIR: coefficients split into float4 pairs
    bool pair_dirty;             // coefficients changed since they were last split
    // material-table coefficients (thiim_set_material_coeffs)
    bool use_table;              // the sweep reads table rows selected by mat[] instead of coeff[]
    const unsigned char *mat;    // per-cell material id
    const void *table;           // n_mat * nz * 28 complex values, context precision
    int n_mat;
    void *pair_table;            // THIIM_C128_PAIR: the table split into float4 pairs
    size_t pair_table_cap;       // entries allocated in pair_table
    bool pair_table_dirty;       // table set or rebuilt since it was last split
    double *mat_eps;             // device: 2 * THIIM_MAX_MATERIALS, the table builder's permittivities
    bool have_coeffs, have_fields, have_norm;
    int zchunk;                  // planes per CTA of the sweep
    int temporal;                // iterations per launch: 1, or 2 (temporal blocking, THIIM_C64)
    unsigned fp64_int_ops;       // THIIM_C128: binary64 operations run on the integer pipe (THIIM_INT_*)
    double *partials;            // 2 doubles per sweep CTA
    size_t partials_cap;         // in CTAs
    double *norms;               // device: |dF|^2, |F|^2 of the last iteration
    double *power;               // device: 2 doubles, thiim_absorbed_power's result
    double *pml;                 // device: 2*nz absorbing-layer conductivities
    int *flag;                   // device: error flag of the coefficient builder
    // defect-correction state (thiim_mixed_solve)
    void *mix_r[THIIM_N_FIELDS]; // complex64 defect r = F64(x) - x
    // adjoint state (thiim_adjoint_iterate)
    void *adj_lh[6];             // conj(c_h) times the adjoint of H^{n+1/2}, per H split
    void *adj_w[6];              // conj(c_e) times the adjoint of E, per E split
    void *adj_states[THIIM_MAX_ADJOINT_SEGMENT][THIIM_N_FIELDS];  // recomputed iterates
    int adj_cap;                 // complete recomputed-iterate sets allocated
    double *adj_norms;           // device: 2 doubles, thiim_adjoint_steady's convergence check
};


namespace thiim {

bool aligned(const void *p, size_t a);
int tiles_x(const thiim_ctx *c);
int tiles_y(const thiim_ctx *c);
int tile_h(const thiim_ctx *c);
// The plain FP64 sweep on the context's FP64 tile (32 x 16 or 32 x 8, tile_h).
cudaError_t launch_sweep_f64_ctx(const thiim_ctx *c, const SweepArgs &a, dim3 grid);
int default_zchunk(const thiim_ctx *c);
int ensure_partials(thiim_ctx *c, size_t ctas);
// Sum n per-CTA partial pairs in a fixed order into out[0], out[1].
cudaError_t finalize_norms(const double *partials, size_t n, double *out, cudaStream_t s);

}  // namespace thiim
