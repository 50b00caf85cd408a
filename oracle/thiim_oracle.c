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

/* ------------------------------------------------------------------------
 * Adjoint of one iteration (reverse-mode derivative of x^{n+1} = F(x^n)).
 *
 * With H' = T_H H + C_H D^- E + b_H and E' = T_E E + C_E D^+ H' + b_E (each
 * split s: x_s' = t_s x_s + Src_s + sign_s c_s D(F)), and adjoints mu of x^{n+1}
 * (mu = dJ/d conj(x), any fixed real multiple), the reverse iteration is
 *   lh_s  = mu_Hs + sum over E splits e reading H component a(s):
 *              sign_e (D^+_{d(e)})^T (conj(c_e) mu_e)
 *   lam_Hs = conj(t_s) lh_s                                   (H, iterate n)
 *   lam_Es = conj(t_s) mu_Es + sum over H splits h reading E component a(s):
 *              sign_h (D^-_{d(h)})^T (conj(c_h) lh_h)         (E, iterate n)
 * with (D^+)^T g = -D^- g and (D^-)^T g = -D^+ g (zero or periodic edges as in
 * the forward).  The coefficient gradients, accumulated with +=, are
 *   H split h:  g_t += lh_h conj(H_h^n),  g_c += lh_h conj(sign_h D^-_{d(h)} E^n),
 *               g_Src += lh_h (Hxy, Hyx)
 *   E split e:  g_t += mu_e conj(E_e^n),  g_c += mu_e conj(sign_e D^+_{d(e)} H^{n+1/2}),
 *               g_Src += mu_e (Exy, Eyx)
 * where H^{n+1/2} is the H part of x^{n+1}.
 * ------------------------------------------------------------------------ */

/* value of array a at (i, j, k) with the boundary rule; zero outside */
static cplx at(const cplx *a, long i, long j, long k, int nx, int ny, int nz, unsigned bc)
{
    if (i < 0 || i >= nx) { if (!(bc & 1u)) return 0; i = (i + nx) % nx; }
    if (j < 0 || j >= ny) { if (!(bc & 2u)) return 0; j = (j + ny) % ny; }
    if (k < 0 || k >= nz) { if (!(bc & 4u)) return 0; k = (k + nz) % nz; }
    return a[((size_t)k * ny + j) * nx + i];
}

int oracle_adjoint_step(int nx, int ny, int nz, unsigned bc, cplx *const *lam, cplx *const *grad,
                        cplx *const *x_n, cplx *const *x_np1, cplx *const *co)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
    const size_t n = (size_t)nx * ny * nz;
    cplx *w[12], *lh[6];
    for (int s = 0; s < 12; s++) w[s] = NULL;
    for (int s = 0; s < 6; s++) lh[s] = NULL;
    int ok = 1;
    for (int s = 6; s < 12; s++) ok &= (w[s] = (cplx *)calloc(n, sizeof(cplx))) != NULL;
    for (int s = 0; s < 6; s++) ok &= (lh[s] = (cplx *)calloc(n, sizeof(cplx))) != NULL;
    if (!ok) goto fail;

    /* w_e = conj(c_e) mu_e for the six E splits */
    for (int e = 6; e < 12; e++)
        for (size_t p = 0; p < n; p++) w[e][p] = conj(co[12 + e][p]) * lam[e][p];

    /* lh_h = mu_h + sum_e sign_e (-(D^-_{d(e)} w_e)), over E splits e whose source
     * component contains h */
    for (int h = 0; h < 6; h++) {
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    size_t p = ((size_t)k * ny + j) * nx + i;
                    cplx acc = lam[h][p];
                    for (int e = 6; e < 12; e++) {
                        const split_rule r = RULES[e];
                        if (r.src_a != h && r.src_b != h) continue;
                        const int ox = r.d == DX, oy = r.d == DY, oz = r.d == DZ;
                        cplx dm = at(w[e], i, j, k, nx, ny, nz, bc) - at(w[e], i - ox, j - oy, k - oz, nx, ny, nz, bc);
                        acc += (double)r.sign * (-dm);
                    }
                    lh[h][p] = acc;
                }
    }
    /* H gradients (need E^n differences) and lambda_H */
    for (int h = 0; h < 6; h++) {
        const split_rule r = RULES[h];
        const int ox = r.d == DX, oy = r.d == DY, oz = r.d == DZ;
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    size_t p = ((size_t)k * ny + j) * nx + i;
                    cplx D = full_at(x_n, r.src_a, r.src_b, i, j, k, nx, ny, nz, bc) -
                             full_at(x_n, r.src_a, r.src_b, i - ox, j - oy, k - oz, nx, ny, nz, bc);
                    grad[h][p] += lh[h][p] * conj(x_n[h][p]);
                    grad[12 + h][p] += lh[h][p] * conj((double)r.sign * D);
                    if (r.src_arr >= 0) grad[r.src_arr][p] += lh[h][p];
                }
    }
    /* lambda_E = conj(t_e) mu_e + sum_h sign_h (-(D^+_{d(h)} v_h)), v_h = conj(c_h) lh_h,
     * over H splits h whose source component contains e; E gradients */
    for (int e = 6; e < 12; e++) {
        const split_rule r = RULES[e];
        const int ox = r.d == DX, oy = r.d == DY, oz = r.d == DZ;
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    size_t p = ((size_t)k * ny + j) * nx + i;
                    cplx mu = lam[e][p];
                    cplx D = full_at(x_np1, r.src_a, r.src_b, i + ox, j + oy, k + oz, nx, ny, nz, bc) -
                             full_at(x_np1, r.src_a, r.src_b, i, j, k, nx, ny, nz, bc);
                    grad[e][p] += mu * conj(x_n[e][p]);
                    grad[12 + e][p] += mu * conj((double)r.sign * D);
                    if (r.src_arr >= 0) grad[r.src_arr][p] += mu;
                    cplx acc = conj(co[e][p]) * mu;
                    for (int h = 0; h < 6; h++) {
                        const split_rule q = RULES[h];
                        if (q.src_a != e && q.src_b != e) continue;
                        const int qx = q.d == DX, qy = q.d == DY, qz = q.d == DZ;
                        /* v_h at (p + e_d) and p */
                        cplx v1 = conj(at(co[12 + h], i + qx, j + qy, k + qz, nx, ny, nz, bc)) *
                                  at(lh[h], i + qx, j + qy, k + qz, nx, ny, nz, bc);
                        cplx v0 = conj(co[12 + h][p]) * lh[h][p];
                        acc += (double)q.sign * (-(v1 - v0));
                    }
                    w[e][p] = acc;          /* new lambda_E, stored after the loop */
                }
    }
    for (int e = 6; e < 12; e++) memcpy(lam[e], w[e], n * sizeof(cplx));
    for (int h = 0; h < 6; h++)
        for (size_t p = 0; p < n; p++) lam[h][p] = conj(co[h][p]) * lh[h][p];
    for (int s = 6; s < 12; s++) free(w[s]);
    for (int s = 0; s < 6; s++) free(lh[s]);
    return 0;
fail:
    for (int s = 6; s < 12; s++) free(w[s]);
    for (int s = 0; s < 6; s++) free(lh[s]);
    return -2;
}
