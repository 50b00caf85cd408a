/*
 * thiim.h — C ABI of the GB300 THIIM E/H sweep library (libthiim.so).
 *
 * The library runs the hot path of the Time Harmonic Inverse Iteration
 * Method (Malas et al., "Optimization of an electromagnetics code with
 * multicore wavefront diamond blocking and multi-dimensional intra-tile
 * parallelization", arXiv 1510.05218): the coupled H-field and E-field update
 * sweeps of Eqs. 3-5 over the staggered Yee grid with the split-field
 * absorbing layer of Eqs. 6-7 (Sec. I-A), whose per-cell data are the 12
 * split field arrays and 28 coefficient arrays of Sec. III.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid:    nx * ny * nz cells; cell (i, j, k) is element (k*ny + j)*nx + i
 *          of every array (x fastest, the layout of Listing 1).
 * Arrays:  contiguous complex values, interleaved (re, im):
 *          THIIM_C128, THIIM_C128_PAIR -> 16-byte double complex, 16-byte aligned;
 *          THIIM_C64                   ->  8-byte float complex,   8-byte aligned.
 * Fields:  12 splits, in this order (split F_ab of component a reads
 *          component b of the other field, as in Listings 1-2):
 *            Hxy Hxz Hyx Hyz Hzx Hzy Exy Exz Eyx Eyz Ezx Ezy
 * Coeffs:  28 arrays: t[12] and c[12] in the field order, then the source
 *          arrays SrcHxy SrcHyx SrcExy SrcEyx (Sec. III: 4*3 + 8*2 = 28).
 * Update:  x_s <- t_s x_s + Src_s + sign_s c_s D_s(F)   (Listings 1-2)
 *          where F is the full component that split s reads (sum of its two
 *          splits), D is a backward difference for H (reads k-1, j-1, i-1)
 *          and a forward difference for E (reads +1), and sign_s is the sign
 *          of the term in the curl:
 *            Hxy +dz Ey  Hxz -dy Ez  Hyx -dz Ex  Hyz +dx Ez  Hzx +dy Ex  Hzy -dx Ey
 *            Exy -dz Hy  Exz +dy Hz  Eyx +dz Hx  Eyz -dx Hz  Ezx -dy Hx  Ezy +dx Hy
 * Order:   one iteration = all six H updates (reading E^n), then all six E
 *          updates (reading the new H), Eqs. 3-4.
 * Bounds:  THIIM_PERIODIC_X/Y/Z wrap the index; a direction without its flag
 *          reads zero outside the grid (homogeneous Dirichlet, Sec. II-B).
 * Memory:  the caller owns every field, coefficient, lambda and gradient
 *          buffer (device memory); the library borrows the pointers until the
 *          next set call or thiim_destroy and owns only its context and
 *          scratch: a second field set of 12 arrays for the out-of-place
 *          sweep, the FP32-pair copy of the coefficients (THIIM_C128_PAIR),
 *          the work arrays of the adjoint and defect-correction calls when
 *          those are used, and a few kilobytes of reduction partials.
 * Streams: all work is enqueued on the stream given to thiim_create (a
 *          cudaStream_t; NULL = legacy default stream) and returns before it
 *          runs, except calls documented as synchronising.
 * Errors:  every int-returning call returns THIIM_OK (0) or a negative
 *          thiim_status; no exception or abort crosses the ABI.  A call that
 *          fails leaves the context usable and the fields unchanged unless
 *          stated otherwise.
 */
#ifndef THIIM_H
#define THIIM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct thiim_ctx thiim_ctx;

enum thiim_precision {
    THIIM_C128 = 0,     /* complex128 storage, FP64 arithmetic */
    THIIM_C64 = 1,      /* complex64 storage, FP32 arithmetic */
    THIIM_C128_PAIR = 2 /* complex128 storage, arithmetic on FP32 pairs
                           (hi + lo, ~2^-48 relative per operation) */
};

enum thiim_bc_flags {
    THIIM_PERIODIC_X = 1u,
    THIIM_PERIODIC_Y = 2u,
    THIIM_PERIODIC_Z = 4u
};

enum thiim_status {
    THIIM_OK = 0,
    THIIM_ERR_ARG = -1,       /* bad size, count, flag or NULL pointer */
    THIIM_ERR_ALIGN = -2,     /* an array is not aligned to its element size */
    THIIM_ERR_STATE = -3,     /* call order violated (e.g. iterate before set_fields) */
    THIIM_ERR_CUDA = -4,      /* a CUDA runtime call or kernel launch failed */
    THIIM_ERR_TIMEOUT = -5,   /* a bounded device-side wait expired */
    THIIM_ERR_NONFINITE = -6, /* a reduction saw NaN or Inf */
    THIIM_ERR_NOMEM = -7      /* the library could not allocate its scratch */
};

/* Binary64 operations of the THIIM_C128 sweep that may run on the integer
 * pipe (thiim_set_fp64_int_ops). */
enum thiim_int_ops {
    THIIM_INT_ADD = 1u,   /* additions and subtractions */
    THIIM_INT_MUL = 2u,   /* the leading product t * x of the updates without a source */
    THIIM_INT_SUMS = 4u   /* only the additions forming the full-field sums (not the differences) */
};

/* Number of field / coefficient arrays (Sec. III). */
#define THIIM_N_FIELDS 12
#define THIIM_N_COEFFS 28
/* Longest segment thiim_adjoint_iterate recomputes from one checkpoint. */
#define THIIM_MAX_ADJOINT_SEGMENT 64
/* Materials a coefficient table may hold (the material id is one byte). */
#define THIIM_MAX_MATERIALS 256

/*
 * thiim_create — make a context for an nx * ny * nz grid.
 *   precision: enum thiim_precision.
 *   bc_flags:  OR of enum thiim_bc_flags (the stack workloads use X|Y,
 *              Dirichlet in z behind the absorbing layers, Sec. I-A).
 *   cuda_stream: cudaStream_t on which every later call enqueues its work.
 * *out receives the context.  Errors: THIIM_ERR_ARG for sizes < 1, a cell
 * count above 2^40, an unknown precision or flag; THIIM_ERR_CUDA if the
 * device cannot be queried.  Allocates only the context itself.
 */
int thiim_create(thiim_ctx **out, int nx, int ny, int nz, int precision,
                 unsigned bc_flags, void *cuda_stream);

/* Replace the stream used by later calls. */
int thiim_set_stream(thiim_ctx *ctx, void *cuda_stream);

/*
 * thiim_set_tuning — execution parameters of thiim_iterate (results do not
 * depend on them; the autotuner in paper_1510_05218_gb300/tuning.py picks
 * them by timing candidates that a footprint model admits).
 *   temporal_block: iterations fused per pass over HBM: 1, or 2 for a
 *                   THIIM_C64 context (temporal blocking: each CTA runs two
 *                   staged iterations with a one-plane lag, keeping the
 *                   intermediate iterate in shared memory; bit-identical to
 *                   two single iterations).
 *   zchunk:         z planes per CTA (0 = the library's default).
 * Errors: THIIM_ERR_ARG.
 */
int thiim_set_tuning(thiim_ctx *ctx, int temporal_block, int zchunk);

/*
 * thiim_set_fp64_int_ops — where the THIIM_C128 sweep of thiim_iterate
 * computes its binary64 additions and multiplications (not in the paper; an
 * execution choice for GB300).  Every update of Eqs. 3-5 is the same sequence
 * of IEEE 754 binary64 operations (round to nearest even) whatever is chosen,
 * so the results are bit-identical (NaN payloads aside).  GB300 retires
 * FP64-pipe instructions at ~1.7 per SM and clock and integer instructions at
 * 64-128, so the FP64 sweep is bound by its FP64 pipe; THIIM_INT_ADD computes
 * the additions exactly in integer arithmetic instead (every operand pair,
 * without branches), THIIM_INT_SUMS only those forming the full-field sums,
 * THIIM_INT_MUL the leading products (normal operands and results; the rest
 * on the FP64 pipe).  The fused multiply-adds always use the FP64 pipe.  Measured on GB300 the sweep is not faster with either (an
 * integer addition costs ~75 integer instructions), so the default is 0.
 *   ops: 0 (everything on the FP64 pipe, the default), THIIM_INT_ADD,
 *        THIIM_INT_ADD | THIIM_INT_MUL, or THIIM_INT_SUMS.
 * Errors: THIIM_ERR_ARG (not a THIIM_C128 context, other values).
 */
int thiim_set_fp64_int_ops(thiim_ctx *ctx, unsigned ops);

/*
 * thiim_set_coeffs — borrow the 28 coefficient arrays (device pointers, in the
 * context's precision, layout above).  Errors: THIIM_ERR_ARG on NULL,
 * THIIM_ERR_ALIGN on misalignment.
 * THIIM_C128_PAIR: the next thiim_iterate splits the coefficients into FP32
 * pairs held by the library (28 more arrays of the same size) and reuses the
 * split until thiim_set_coeffs or thiim_build_coeffs is called again; call
 * one of them after changing the arrays' contents.
 */
int thiim_set_coeffs(thiim_ctx *ctx, void *const coeff[THIIM_N_COEFFS]);

/*
 * thiim_set_fields — borrow the 12 field arrays (device pointers).  They hold
 * the current iterate x^n and are updated in place by thiim_iterate.  The
 * first call allocates the library's second field set (12 arrays of the same
 * size) used by the out-of-place sweep; THIIM_ERR_NOMEM if that fails.
 */
int thiim_set_fields(thiim_ctx *ctx, void *const field[THIIM_N_FIELDS]);

/*
 * thiim_iterate — enqueue n_iters THIIM iterations (Eqs. 3-5): each is the
 * six H half-step updates followed by the six E updates.  When it completes
 * on the stream, the caller's field arrays hold x^{n + n_iters}.  Under
 * THIIM_C128_PAIR the intermediate iterates of one call are kept as FP32
 * pairs (in the caller's and the library's field arrays) and only the final
 * one is written as complex128.  The last
 * iteration also accumulates the norms that thiim_residual reports (per
 * thread in FP64, or in FP32 pairs, ~48 bits, under THIIM_C128_PAIR; summed
 * across threads and CTAs in FP64).
 * n_iters = 0 does nothing.  Errors: THIIM_ERR_STATE if fields or
 * coefficients are missing, THIIM_ERR_ARG if n_iters < 0 or the grid needs
 * more CTAs than one launch takes (2^31 - 1 tiles, or 65535 z chunks: raise
 * zchunk with thiim_set_tuning), THIIM_ERR_CUDA.
 */
int thiim_iterate(thiim_ctx *ctx, int n_iters);

/*
 * thiim_residual — synchronises the stream and returns in *rel_residual the
 * relative update of the most recent iteration run by thiim_iterate,
 *   || F^{n} - F^{n-1} ||_2 / || F^{n} ||_2,
 * over the six full field components F (Ex = Exy + Exz, ..., Hz = Hzx + Hzy)
 * of every cell, accumulated in FP64.  (The split parts alone do not settle
 * where sigma* = 0: their difference is not driven, so the full fields are
 * the converging quantity.)  Returns 0 in *rel_residual when F^n = 0.
 * The sums are formed per CTA tile and then over the tiles in a fixed order,
 * so a result repeats bit for bit on the same grid; the FP64 sweep's tile is
 * 32 x 16 cells on grids of at least 2^23 cells and 32 x 8 below, the same
 * for all its variants (coefficient table, integer-pipe operations).
 * Errors: THIIM_ERR_STATE if no iteration ran since set_fields,
 * THIIM_ERR_NONFINITE if a norm is NaN or Inf, THIIM_ERR_CUDA.
 */
int thiim_residual(thiim_ctx *ctx, double *rel_residual);

/*
 * thiim_build_coeffs — fill the 28 coefficient arrays of a layered problem
 * from per-cell material data, in the context's precision (the discrete
 * Eqs. 3-5 solved for the new value; Eq. 5 where Re(eps_r) < 0):
 *   eps_r:       device array of nx*ny*nz complex128 relative permittivities
 *                in the physics convention (Im > 0 lossy); the paper's fields
 *                vary as e^{+i omega t}, so the material conductivity is
 *                sigma = omega * Im(eps_r) and eps = Re(eps_r).  mu = 1.
 *   sigma_pml_e: host array of nz absorbing-layer conductivities at the E
 *                planes (z = k); added to the four splits that difference
 *                along z (Hxy, Hyx, Exy, Eyx) — for H from sigma_pml_h
 *                (H plane k sits at z = k - 1/2).  NULL = none.
 *   omega, tau:  frequency and pseudo time step (tau > 0).
 *   k_s, amp:    plane-wave source: an x-polarised wave of complex amplitude
 *                (amp_re, amp_im) enters at the total-field/scattered-field
 *                plane k_s (E planes >= k_s and H planes > k_s are total
 *                field); k_s < 0 means no source (all Src arrays zero).
 *   coeff:       28 device arrays (may equal those given to set_coeffs).
 * Errors: THIIM_ERR_ARG (NULL, tau <= 0, k_s >= nz, omega tau beyond the
 * discrete dispersion range), THIIM_ERR_ALIGN, THIIM_ERR_CUDA.
 */
int thiim_build_coeffs(thiim_ctx *ctx, const void *eps_r,
                       const double *sigma_pml_e, const double *sigma_pml_h,
                       double omega, double tau, int k_s, double amp_re,
                       double amp_im, void *const coeff[THIIM_N_COEFFS]);

/*
 * thiim_build_coeffs_jones — thiim_build_coeffs for a normally incident wave
 * of any polarisation.  The paper covers a solar cell's spectrum with 80-160
 * runs (Sec. V); an unpolarised spectrum averages the x- and y-polarised
 * runs.  jones: host array {Re A_x, Im A_x, Re A_y, Im A_y}, the incident
 * E = (A_x, A_y, 0) at plane k_s.  The y component (E_y, H_x = +dE_y/(i
 * omega_t)) enters through the two Src arrays the x-polarised wave leaves
 * zero: SrcHxy(k_s) = -c_Hxy A_y, SrcEyx(k_s) = -c_Eyx H_x,inc(k_s).
 * thiim_build_coeffs(..., amp_re, amp_im, ...) equals jones = {amp_re,
 * amp_im, 0, 0}.  Errors as thiim_build_coeffs, plus THIIM_ERR_ARG for a
 * NULL or non-finite jones.
 */
int thiim_build_coeffs_jones(thiim_ctx *ctx, const void *eps_r,
                             const double *sigma_pml_e, const double *sigma_pml_h,
                             double omega, double tau, int k_s, const double jones[4],
                             void *const coeff[THIIM_N_COEFFS]);

/*
 * thiim_absorbed_power — P = 1/2 sum over cells of sigma |E|^2 for the
 * context's current fields (E = the full components, split sums), summed in
 * FP64 in a fixed order (deterministic).  At the fixed point the power
 * dissipated in those cells is cos(omega tau / 2) P (the loss term of Eqs. 3
 * and 5 carries the phase e^{+-i omega tau/2}); over the incident power of
 * the plane wave that is the absorption of a solar cell at one wavelength
 * and polarisation, the quantity of the paper's spectrum runs (Sec. V).
 *   sigma: device array of nx*ny*nz conductivities (layout as the fields),
 *          e.g. omega Im(eps_r) on the absorbing layer and 0 elsewhere.
 *   power: host double receiving P.
 * Synchronises the stream.  Errors: THIIM_ERR_ARG (NULL), THIIM_ERR_ALIGN
 * (sigma not 8-byte aligned), THIIM_ERR_STATE (no fields set),
 * THIIM_ERR_NONFINITE, THIIM_ERR_NOMEM, THIIM_ERR_CUDA.
 */
int thiim_absorbed_power(thiim_ctx *ctx, const double *sigma, double *power);

/*
 * Compressed coefficients (a variant; the paper stores all 28 arrays, Sec.
 * III, 40 complex values per cell in total).  In the workloads of Sec. I-A a
 * cell's coefficients depend only on its material (eps_r) and its plane
 * (absorbing-layer conductivity, source plane), so they can be kept as a
 * table with one row of 28 per (material, plane) and a one-byte material id
 * per cell: about 1 byte of coefficient data per cell instead of 28 complex
 * values.  The sweep reads row (mat[p], k) where it would read element p of
 * the 28 arrays; the arithmetic is otherwise the same, so a table built by
 * thiim_build_material_table gives results bit-identical to the arrays that
 * thiim_build_coeffs builds from the same materials.
 *
 * thiim_build_material_table — fill the table of n_mat materials.
 *   n_mat:   1 .. THIIM_MAX_MATERIALS.
 *   eps_mat: host array of 2 * n_mat doubles, (Re, Im) of each material's
 *            relative permittivity, conventions as in thiim_build_coeffs.
 *   jones:   host array {Re A_x, Im A_x, Re A_y, Im A_y} of the plane wave
 *            (as in thiim_build_coeffs_jones).
 *   the others as in thiim_build_coeffs.
 *   table:   device array of n_mat * nz * 28 complex values in the context's
 *            precision (complex64 for THIIM_C64, else complex128); entry
 *            ci of row (m, k) is at table[(m * nz + k) * 28 + ci], ci in the
 *            coefficient order of thiim_set_coeffs.  Owned by the caller.
 * Synchronises the stream.  Errors: THIIM_ERR_ARG (as thiim_build_coeffs;
 * also n_mat out of range or a zero or non-finite permittivity),
 * THIIM_ERR_ALIGN, THIIM_ERR_NOMEM, THIIM_ERR_CUDA.  n_mat * nz above 2^31 - 1
 * is rejected with THIIM_ERR_ARG.
 */
int thiim_build_material_table(thiim_ctx *ctx, int n_mat, const double *eps_mat,
                               const double *sigma_pml_e, const double *sigma_pml_h,
                               double omega, double tau, int k_s, const double jones[4],
                               void *table);

/*
 * thiim_set_material_coeffs — borrow a material map and table in place of
 * the 28 coefficient arrays; thiim_set_coeffs switches back.
 *   mat:   device array of nx*ny*nz material ids (uint8, layout as the
 *          fields), each below n_mat.  Ids are not checked on the device: an
 *          id >= n_mat reads outside the table.
 *   n_mat: rows of the table, 1 .. THIIM_MAX_MATERIALS.
 *   table: device table as filled by thiim_build_material_table.
 * thiim_iterate then runs one iteration per launch (thiim_set_tuning's
 * temporal_block is ignored).  THIIM_C128_PAIR: the next thiim_iterate splits
 * the table into FP32 pairs held by the library; call this function again
 * after changing the table's contents.  thiim_mixed_solve,
 * thiim_batch_iterate and thiim_adjoint_iterate need the 28 arrays and return
 * THIIM_ERR_STATE for a context in this mode.  Errors: THIIM_ERR_ARG,
 * THIIM_ERR_ALIGN.
 */
int thiim_set_material_coeffs(thiim_ctx *ctx, const unsigned char *mat, int n_mat,
                              const void *table);

/*
 * thiim_mixed_solve — complex64 sweeps with FP64 defect correction.
 *   ctx:        a THIIM_C64 context with its complex64 coefficients set
 *               (thiim_set_coeffs / thiim_build_coeffs) and 12 complex64
 *               work arrays given to thiim_set_fields (they receive the
 *               corrections; their contents are overwritten).
 *   coeff64:    the same problem's 28 complex128 coefficient arrays.
 *   x64:        12 complex128 field arrays: the FP64 iterate, updated in place.
 *   Each outer step evaluates the FP64 defect r = F(x) - x (one FP64 sweep
 *   with coeff64; the relative full-field norm ||r|| / ||F(x)|| is the
 *   residual of thiim_residual), stops if it is <= tol, otherwise advances
 *   the correction inner_iters times by delta <- M32 delta + r (complex64,
 *   FP32 arithmetic, delta starting at 0) and sets x += delta.  In exact
 *   arithmetic one outer step equals inner_iters plain iterations.  At most
 *   max_outer corrections are applied; the defect is evaluated once more
 *   after the last one.  Synchronises the stream once per outer step.
 *   *outer_done: corrections applied; *rel_residual: last defect residual.
 *   Allocates 12 complex64 arrays for r on the first call.
 * Errors: THIIM_ERR_ARG (not a THIIM_C64 context, inner_iters < 1, NULL),
 * THIIM_ERR_STATE, THIIM_ERR_ALIGN, THIIM_ERR_NOMEM, THIIM_ERR_NONFINITE,
 * THIIM_ERR_CUDA.
 */
int thiim_mixed_solve(thiim_ctx *ctx, void *const coeff64[THIIM_N_COEFFS],
                      void *const x64[THIIM_N_FIELDS], int inner_iters, int max_outer,
                      double tol, int *outer_done, double *rel_residual);

/*
 * thiim_adjoint_iterate — reverse n_back iterations (adjoint / reverse-mode
 * derivative of x^{n} = F^{n_back}(x^{n0}), n = n0 + n_back).  Not in the
 * paper; it turns the sweep into a differentiable solver.
 *   ctx:            THIIM_C128 context with coefficients set.
 *   lambda:         12 complex128 arrays: on entry the adjoint of x^{n}
 *                   (the gradient of a real objective J with respect to
 *                   conj(x), times any fixed real factor — e.g. torch's
 *                   complex gradient, which is 2 dJ/dconj(x)); on return the
 *                   adjoint of x^{n0}, in place.
 *   grad_coeff:     28 complex128 arrays; the same-convention gradients of J
 *                   with respect to each coefficient array are ADDED to them.
 *   fwd_checkpoint: the forward iterate x^{n0} (12 complex128 arrays, read
 *                   only).  The library recomputes x^{n0+1} .. x^{n} from it
 *                   with the FP64 sweep into its own scratch (n_back field
 *                   sets, kept for later calls), then runs the n_back reverse
 *                   steps: per step one kernel for the H part and one for the
 *                   E part (see csrc/thiim_adjoint.cu for the formulas).
 *   n_back:         1 .. THIIM_MAX_ADJOINT_SEGMENT.
 * Enqueued on the context's stream.  Errors: THIIM_ERR_ARG (not a
 * THIIM_C128 context, bad n_back, NULL), THIIM_ERR_ALIGN, THIIM_ERR_STATE,
 * THIIM_ERR_NOMEM, THIIM_ERR_CUDA.
 */
int thiim_adjoint_iterate(thiim_ctx *ctx, void *const lambda[THIIM_N_FIELDS],
                          void *const grad_coeff[THIIM_N_COEFFS],
                          const void *const fwd_checkpoint[THIIM_N_FIELDS], int n_back);

/*
 * thiim_adjoint_steady — reverse-mode gradient of an objective of the
 * CONVERGED solution (not in the paper; inverse design of the converged
 * absorption).  At a fixed point x* = F(x*) of the iteration the gradient of
 * J(x*) with respect to the coefficients is (dF/da)^H lam*, where the
 * adjoint field lam* = M^H lam* + g solves the adjoint fixed point (M the
 * linear part of one iteration, g the gradient of J with respect to conj(x*)
 * in torch's convention).  lam* = sum_k (M^H)^k g is summed term by term with
 * the reverse iteration of thiim_adjoint_iterate (without gradient work per
 * term), and the coefficient gradient is evaluated once, on lam*.
 *   ctx:         a THIIM_C128 context with its 28 coefficient arrays set.
 *   lambda:      12 device arrays; in: g; out: lam* (the terms summed).
 *   grad_coeff:  28 device arrays; the gradient is ADDED to them.
 *   x_star:      12 device arrays, the converged iterate (read only).
 *   max_iters:   maximum number of terms (>= 1; 1 gives the one-term sum g).
 *   check_every: terms between convergence checks (>= 1; each synchronises).
 *   tol:         stop once |last term| <= tol |lam*| (norms over the 12
 *                arrays); 0 sums exactly max_iters terms.
 *   iters_out, rel_out: optional; terms summed, |last term| / |lam*|.
 * Convergence: the iteration has modes that never decay where sigma* = 0
 * (split differences and curl-free H rotate with |t| = 1); sources never
 * excite them, so the forward solve converges, but a seed g with an
 * antisymmetric part on an E split pair, or a curl-free part on H, feeds
 * them and the sum does not converge (rel_out stays large).  An objective
 * of the full E components (g equal on the two splits of each E component,
 * zero on H), such as the absorbed power, never does.  Scratch: 18 complex128 arrays of the grid
 * (shared with thiim_adjoint_iterate).  Synchronises the stream.
 * Errors: THIIM_ERR_ARG, THIIM_ERR_ALIGN, THIIM_ERR_STATE, THIIM_ERR_NOMEM,
 * THIIM_ERR_NONFINITE, THIIM_ERR_CUDA.
 */
int thiim_adjoint_steady(thiim_ctx *ctx, void *const lambda[THIIM_N_FIELDS],
                         void *const grad_coeff[THIIM_N_COEFFS],
                         const void *const x_star[THIIM_N_FIELDS], int max_iters, int check_every,
                         double tol, int *iters_out, double *rel_out);

/*
 * thiim_build_coeffs_grad — chain rule through thiim_build_coeffs: given the
 * gradients G_a of a real objective with respect to the 28 complex128
 * coefficient arrays (torch's complex convention, 2 dJ/dconj(a)), write
 *   grad_eps_re[p] = dJ / d Re(eps_r[p]) = Re sum_a conj(G_a[p]) d a[p] / d Re(eps_r[p])
 * for every cell (device array of nx*ny*nz doubles), holding Im(eps_r) and
 * hence the material conductivity fixed.  Only the six E splits' t and c (and
 * SrcExy at the source plane) depend on the permittivity (Eqs. 3 and 5).
 * The other arguments are those given to thiim_build_coeffs (sigma_pml_h is
 * not needed); the source term is that of its x-polarised wave (the y part
 * of thiim_build_coeffs_jones, SrcEyx, is not differentiated here).
 * Enqueued on the context's stream.
 * Errors: THIIM_ERR_ARG, THIIM_ERR_ALIGN, THIIM_ERR_NOMEM, THIIM_ERR_CUDA.
 */
int thiim_build_coeffs_grad(thiim_ctx *ctx, const void *eps_r, const double *sigma_pml_e,
                            double omega, double tau, int k_s, double amp_re, double amp_im,
                            const void *const grad_coeff[THIIM_N_COEFFS], double *grad_eps_re);

/*
 * thiim_batch_iterate — advance nb independent solves together.
 *   ctx[0..nb-1]: contexts of one precision on one device, each with fields
 *                 and coefficients set; grids may differ in size.
 *   Every iteration of all still-active solves is ONE persistent launch that
 *   walks a list of (solve, tile column, z chunk) items; check_every
 *   iterations (even, >= 2) and the per-solve residual run as one captured
 *   CUDA graph, after which solves whose residual (as thiim_residual) is
 *   <= tol, or which reached max_iters, leave the batch.
 *   All work runs on ctx[0]'s stream; the call synchronises it after each
 *   chunk and at the end.  On return every solve's arrays hold its final
 *   iterate (complex128 / complex64), thiim_residual(ctx[b]) reports its last
 *   residual, iters_out[b] (optional) the iterations it ran and
 *   residual_out[b] (optional) the residual.  Temporary device memory for the
 *   item list and partial norms is allocated per call.
 * Errors: THIIM_ERR_ARG (mixed precisions or devices, check_every odd or < 2),
 * THIIM_ERR_STATE, THIIM_ERR_NOMEM, THIIM_ERR_NONFINITE, THIIM_ERR_CUDA.
 */
int thiim_batch_iterate(thiim_ctx *const ctx[], int nb, int max_iters, int check_every,
                        double tol, int *iters_out, double *residual_out);

/*
 * thiim_step_noalloc — one THIIM iteration that allocates no memory.
 *   For callers that cannot call cudaMalloc (code running under another
 *   framework's memory pool or allocator hooks, or with all device memory
 *   reserved up front).  The paper has no counterpart; this is a deployment
 *   variant of thiim_iterate for a single iteration.
 *   src: 12 field arrays holding x^n (read only); dst: 12 other field arrays
 *   that receive x^{n+1} (no array may appear in both); coeff: 28 arrays;
 *   all device pointers in the layout above.  cuda_stream: cudaStream_t.
 *   rel_residual: if non-NULL, the call synchronises the stream and returns
 *   the relative full-field update of this iteration (as thiim_residual);
 *   if NULL, the call only enqueues the sweep and returns.
 *   Scratch: the reduction partials live in one fixed device array of
 *   16384 CTAs x 16 B (+16 B) = 256 KiB, defined in the library and held by
 *   every GPU that loads it until the process exits.  A grid needing more
 *   than 16384 CTAs of 32 x 8 cells (ceil(nx/32) * ceil(ny/8) > 16384) is
 *   rejected with THIIM_ERR_ARG before anything is enqueued.  Each call with
 *   a residual looks up the array's device address (the first lookup on a
 *   device loads the library's device code: make that first call before any
 *   stream capture).  All calls
 *   share the array, so calls whose GPU work overlaps (other streams or
 *   host threads on the same device) race on it.
 * Errors: THIIM_ERR_ARG, THIIM_ERR_ALIGN, THIIM_ERR_CUDA, THIIM_ERR_NONFINITE.
 */
int thiim_step_noalloc(int nx, int ny, int nz, int precision, unsigned bc_flags,
                       void *const src[THIIM_N_FIELDS], void *const dst[THIIM_N_FIELDS],
                       void *const coeff[THIIM_N_COEFFS], void *cuda_stream,
                       double *rel_residual);

/*
 * thiim_fp64_pipe_rate — measure the FP64 fused multiply-add throughput of
 * the current device (a measurement helper; the paper has no counterpart).
 * GB300 runs FP64 at a small fraction of its FP32 rate, so the FP64 sweep can
 * be bound by that pipe instead of by memory bandwidth (the paper's Eqs. 8-10
 * model only memory); this gives the denominator of that roofline, measured
 * at the clocks of the caller's run.  A grid of 8 CTAs per SM runs 8
 * independent FMA chains per thread; the best of 5 timed launches on
 * cuda_stream (a cudaStream_t) is reported.
 *   fma_per_s: host double receiving FP64 FMA instructions per second,
 *              device-wide (one FMA = one FP64 pipe slot; DADD and DMUL take
 *              one slot each as well).
 * Allocates and frees a few kilobytes; synchronises the stream.
 * Errors: THIIM_ERR_ARG (NULL), THIIM_ERR_NOMEM, THIIM_ERR_CUDA.
 */
int thiim_fp64_pipe_rate(void *cuda_stream, double *fma_per_s);

/* Release the context and its scratch (synchronises the stream first). */
void thiim_destroy(thiim_ctx *ctx);

/* Static, human-readable text of a thiim_status code. */
const char *thiim_strerror(int status);

/* Library version as major*10000 + minor*100 + patch. */
int thiim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* THIIM_H */
