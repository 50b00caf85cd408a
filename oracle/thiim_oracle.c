/*
 * THIIM E/H sweep oracle: plain, slow, FP64 C.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; it exists so that tests, the smoke check and the CPU
 * baseline timing have an independent reference for the GPU kernels.
 *
 * What it computes (paper Sec. I-A, Eqs. 3-7; Sec. III, Listings 1-2):
 *   one THIIM iteration = the six H split updates (Eq. 4), each reading the
 *   full E of the previous iterate, followed by the six E split updates
 *   (Eq. 3, or Eq. 5 where eps < 0, already folded into the coefficients),
 *   each reading the new H.  Every split s is updated by
 *       x_s <- t_s * x_s + Src_s + sign_s * c_s * D_d(s)(F_src(s))
 *   where F_src(s) is the sum of the two splits of the other field's vector
 *   component that s reads, D is a backward difference for H (Listing 1 reads
 *   k and k-1; Listing 2 reads j-1 and j) and a forward difference for E
 *   (E reads H at +1, Fig. 3).  Listing 1 (H_yx) has sign -1 with a z
 *   difference and a source array; Listing 2 (H_zx) has sign +1 with a y
 *   difference, written there as -c*(F(j-1) - F(j)).
 *
 * Layout (Listing 1): array[(k*Ny + j)*Nx + i], x fastest, double complex.
 * Field order:  Hxy Hxz Hyx Hyz Hzx Hzy Exy Exz Eyx Eyz Ezx Ezy
 * Coefficients: t[12] (same order), c[12] (same order),
 *               SrcHxy, SrcHyx, SrcExy, SrcEyx.
 * Boundaries: bit 0 periodic x, bit 1 periodic y, bit 2 periodic z; a
 * non-periodic direction reads zero outside the grid (homogeneous Dirichlet,
 * the benchmark boundary of Sec. II-B).
 *
 * Each split is its own loop nest over k, j, i, as in the paper's naive code
 * (Sec. III-A); there is no blocking, fusion or reordering.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { DX = 0, DY = 1, DZ = 2 };

/* One row of the split table: derivative direction, the two splits whose sum
 * is the full component read, the sign of the curl term, the source array. */
typedef struct {
    int d;
    int src_a, src_b;
    int sign;
    int src_arr; /* index into the 28 coefficients, or -1 */
} split_rule;

/* Indices of the split fields. */
enum { HXY, HXZ, HYX, HYZ, HZX, HZY, EXY, EXZ, EYX, EYZ, EZX, EZY };

/* -curl E for H (Eq. 4, Eqs. 6-7 split):
 *   (-curl E)_x = dE_y/dz - dE_z/dy ; (-curl E)_y = dE_z/dx - dE_x/dz ;
 *   (-curl E)_z = dE_x/dy - dE_y/dx
 * +curl H for E (Eq. 3):
 *   (curl H)_x = dH_z/dy - dH_y/dz ; (curl H)_y = dH_x/dz - dH_z/dx ;
 *   (curl H)_z = dH_y/dx - dH_x/dy                                          */
static const split_rule RULES[12] = {
    /* Hxy */ {DZ, EYX, EYZ, +1, 24},
    /* Hxz */ {DY, EZX, EZY, -1, -1},
    /* Hyx */ {DZ, EXY, EXZ, -1, 25},
    /* Hyz */ {DX, EZX, EZY, +1, -1},
    /* Hzx */ {DY, EXY, EXZ, +1, -1},
    /* Hzy */ {DX, EYX, EYZ, -1, -1},
    /* Exy */ {DZ, HYX, HYZ, -1, 26},
    /* Exz */ {DY, HZX, HZY, +1, -1},
    /* Eyx */ {DZ, HXY, HXZ, +1, 27},
    /* Eyz */ {DX, HZX, HZY, -1, -1},
    /* Ezx */ {DY, HXY, HXZ, -1, -1},
    /* Ezy */ {DX, HYX, HYZ, +1, -1},
};

/* Full component F_a + F_b at (i, j, k); zero outside a non-periodic edge. */
static cplx full_at(cplx *const *f, int a, int b, long i, long j, long k,
                    int nx, int ny, int nz, unsigned bc)
{
    if (i < 0 || i >= nx) { if (!(bc & 1u)) return 0; i = (i + nx) % nx; }
    if (j < 0 || j >= ny) { if (!(bc & 2u)) return 0; j = (j + ny) % ny; }
    if (k < 0 || k >= nz) { if (!(bc & 4u)) return 0; k = (k + nz) % nz; }
    size_t p = ((size_t)k * ny + j) * nx + i;
    return f[a][p] + f[b][p];
}

/* Update split s in place.  backward != 0: D = F(p) - F(p - e_d) (H);
 * otherwise D = F(p + e_d) - F(p) (E).  Accumulates |x_new - x_old|^2 and
 * |x_new|^2 into *dn2 / *xn2. */
static void update_split(int s, int nx, int ny, int nz, unsigned bc,
                         cplx *const *f, cplx *const *co, int backward,
                         double *dn2, double *xn2, int nthreads)
{
    const split_rule r = RULES[s];
    const int ox = r.d == DX, oy = r.d == DY, oz = r.d == DZ;
    cplx *x = f[s];
    const cplx *t = co[s];
    const cplx *c = co[12 + s];
    const cplx *src = r.src_arr >= 0 ? co[r.src_arr] : NULL;
    double d_acc = 0.0, x_acc = 0.0;
#pragma omp parallel for num_threads(nthreads) reduction(+ : d_acc, x_acc) schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t p = ((size_t)k * ny + j) * nx + i;
                cplx here = full_at(f, r.src_a, r.src_b, i, j, k, nx, ny, nz, bc);
                cplx D;
                if (backward)
                    D = here - full_at(f, r.src_a, r.src_b, i - ox, j - oy, k - oz, nx, ny, nz, bc);
                else
                    D = full_at(f, r.src_a, r.src_b, i + ox, j + oy, k + oz, nx, ny, nz, bc) - here;
                cplx xn = t[p] * x[p] + (double)r.sign * c[p] * D;
                if (src) xn += src[p];
                cplx dd = xn - x[p];
                d_acc += creal(dd) * creal(dd) + cimag(dd) * cimag(dd);
                x_acc += creal(xn) * creal(xn) + cimag(xn) * cimag(xn);
                x[p] = xn;
            }
    *dn2 += d_acc;
    *xn2 += x_acc;
}

/* n THIIM iterations in place.  On return *rel_change holds
 * ||x^n - x^{n-1}|| / ||x^n|| over all 12 splits (0 if n == 0 or x^n == 0). */
int oracle_iterate(int nx, int ny, int nz, unsigned bc, cplx *const *fields,
                   cplx *const *coeffs, int n, int nthreads, double *rel_change)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || n < 0 || nthreads < 1) return -1;
    double dn2 = 0.0, xn2 = 0.0;
    for (int it = 0; it < n; it++) {
        dn2 = 0.0;
        xn2 = 0.0;
        for (int s = HXY; s <= HZY; s++) update_split(s, nx, ny, nz, bc, fields, coeffs, 1, &dn2, &xn2, nthreads);
        for (int s = EXY; s <= EZY; s++) update_split(s, nx, ny, nz, bc, fields, coeffs, 0, &dn2, &xn2, nthreads);
    }
    if (rel_change) *rel_change = (n > 0 && xn2 > 0.0) ? sqrt(dn2 / xn2) : 0.0;
    return 0;
}

/* Sign, direction and source index of split s (for host-side helpers). */
int oracle_rule(int s, int *d, int *src_a, int *src_b, int *sign, int *src_arr)
{
    if (s < 0 || s >= 12) return -1;
    *d = RULES[s].d; *src_a = RULES[s].src_a; *src_b = RULES[s].src_b;
    *sign = RULES[s].sign; *src_arr = RULES[s].src_arr;
    return 0;
}
