// Adjoint of the THIIM iteration and gradients with respect to the
// coefficients and the permittivity (thiim_adjoint_iterate,
// thiim_build_coeffs_grad).  Not in the paper: this makes the sweep usable
// for inverse design (d objective / d permittivity).
//
// One iteration is H' = T_H H + C_H D^- E + b_H followed by
// E' = T_E E + C_E D^+ H' + b_E (per split s: x_s' = t_s x_s + Src_s +
// sign_s c_s D(F), Listings 1-2).  For adjoints mu of x^{n+1} (the gradient
// of a real objective with respect to conj(x), any fixed real multiple) the
// reverse iteration is
//   lh_h   = mu_h + sum_{E splits e reading H component of h} -sign_e D^-_{d(e)} (conj(c_e) mu_e)
//   lam_h  = conj(t_h) lh_h
//   lam_e  = conj(t_e) mu_e + sum_{H splits h reading E component of e} -sign_h D^+_{d(h)} (conj(c_h) lh_h)
// using (D^+)^T = -D^- and (D^-)^T = -D^+ with the forward's edge rules, and
// the coefficient gradients (accumulated)
//   g_t[h] += lh_h conj(H_h^n)   g_c[h] += lh_h conj(sign_h D^-_{d(h)} E^n)   g_Src += lh_h
//   g_t[e] += mu_e conj(E_e^n)   g_c[e] += mu_e conj(sign_e D^+_{d(e)} H^{n+1/2})   g_Src += mu_e.
// Kernel R1 computes lh, lam_H and the H gradients; kernel R2 the new lam_E
// and the E gradients.  Both are gather kernels, one thread per cell, in FP64
// (FP64-pipe bound, like the forward sweep).  The products a difference
// needs at a cell and at its neighbour are formed once per cell: R1 stores
// v_h = conj(c_h) lh_h for R2, and R2 stores w_e = conj(c_e) lam_e for the next
// step's R1 (adjoint_w_kernel forms w from the incoming lam before the first
// step).  Same operations on the same values as forming them where they are
// used, so the results are unchanged, with 96 instead of 120 FP64
// instructions per cell and kernel.
//
// Steady state (thiim_adjoint_steady): at a fixed point x* = F(x*) every
// state of the reverse iteration is x*, so its gradient contributions sum to
// (dF/da)^H lam* with lam* = sum_k (M^H)^k g, the solution of the adjoint
// fixed point lam* = M^H lam* + g.  The contributions are linear in lam, so
// the iteration propagates lam alone (GRAD = false) while adding every new
// term into lam*, and the gradient kernels run once, on lam*.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "thiim_ctx.h"

using namespace thiim;

namespace {

// Split table (same as include/thiim.h): difference direction, the two
// splits of the full component read, the curl sign, the source array or -1.
// A compile-time function: with the split loops unrolled, the directions and
// signs fold into the code (no FP64 multiplication by +-1, constant index
// offsets).
struct Rule { int d, a, b, sign, src; };
__host__ __device__ constexpr Rule rule_of(int s) {
    return s == HXY ? Rule{2, EYX, EYZ, +1, SRC_HXY}
         : s == HXZ ? Rule{1, EZX, EZY, -1, -1}
         : s == HYX ? Rule{2, EXY, EXZ, -1, SRC_HYX}
         : s == HYZ ? Rule{0, EZX, EZY, +1, -1}
         : s == HZX ? Rule{1, EXY, EXZ, +1, -1}
         : s == HZY ? Rule{0, EYX, EYZ, -1, -1}
         : s == EXY ? Rule{2, HYX, HYZ, -1, SRC_EXY}
         : s == EXZ ? Rule{1, HZX, HZY, +1, -1}
         : s == EYX ? Rule{2, HXY, HXZ, +1, SRC_EYX}
         : s == EYZ ? Rule{0, HZX, HZY, -1, -1}
         : s == EZX ? Rule{1, HXY, HXZ, -1, -1}
         :            Rule{0, HYX, HYZ, +1, -1};
}

struct AdjArgs {
    double2 *lam[12];        // in: adjoint of x^{n+1}; out: adjoint of x^n
    double2 *grad[28];       // accumulated (GRAD kernels only)
    const double2 *xn[12];   // x^n (GRAD kernels only)
    const double2 *xn1[12];  // x^{n+1} (GRAD kernels only)
    const double2 *co[28];
    double2 *v[6];           // scratch: conj(c_h) lh_h per H split (lh: adjoint of H^{n+1/2})
    double2 *w[6];           // scratch: conj(c_e) lam_e per E split, for the next H kernel
    double2 *acc[12];        // if acc[0]: acc += the new lam (steady-state sum)
    int nx, ny, nz;
    unsigned bc;
};

__device__ __forceinline__ double2 c2(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return c2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return c2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return c2(s * a.x, s * a.y); }
// sign * a for a compile-time sign of +-1 (a negation, no multiplication)
template <int SIGN>
__device__ __forceinline__ double2 csign(double2 a) { return SIGN > 0 ? a : c2(-a.x, -a.y); }
__device__ __forceinline__ double2 conjmul(double2 a, double2 b) {   // conj(a) * b
    return c2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// Linear index of (i, j, k) shifted by OFF = +-1 along D, or -1 outside a
// non-periodic edge.
template <int D, int OFF>
__device__ __forceinline__ long long shifted(int i, int j, int k, const AdjArgs &a) {
    int q[3] = {i, j, k};
    const int n[3] = {a.nx, a.ny, a.nz};
    q[D] += OFF;
    if (q[D] < 0 || q[D] >= n[D]) {
        if (!(a.bc & (1u << D))) return -1;
        q[D] = OFF < 0 ? q[D] + n[D] : q[D] - n[D];
    }
    return ((long long)q[2] * a.ny + q[1]) * a.nx + q[0];
}

// Contribution of E split E to the H components' adjoint: -sign_e D^-_{d(e)} w_e,
// w_e = conj(c_e) mu_e (formed by the previous E kernel or adjoint_w_kernel).
template <int E>
__device__ __forceinline__ void adj_h_term(const AdjArgs &a, size_t p, int i, int j, int k, double2 A[3]) {
    constexpr Rule r = rule_of(E);
    constexpr int comp = r.a / 2;   // H component read (0 = x, 1 = y, 2 = z)
    const long long q = shifted<r.d, -1>(i, j, k, a);
    const double2 w0 = a.w[E - 6][p];
    const double2 w1 = q < 0 ? c2(0, 0) : a.w[E - 6][q];
    A[comp] = cadd(A[comp], csign<-r.sign>(csub(w0, w1)));
}

template <bool GRAD, int H>
__device__ __forceinline__ void adj_h_split(const AdjArgs &a, size_t p, int i, int j, int k, const double2 A[3]) {
    constexpr Rule r = rule_of(H);
    const double2 lh = cadd(a.lam[H][p], A[H / 2]);
    if (GRAD) {
        // D^- of the full E component this split reads, from x^n
        const long long q = shifted<r.d, -1>(i, j, k, a);
        const double2 f0 = cadd(a.xn[r.a][p], a.xn[r.b][p]);
        const double2 f1 = q < 0 ? c2(0, 0) : cadd(a.xn[r.a][q], a.xn[r.b][q]);
        const double2 dm = csign<r.sign>(csub(f0, f1));
        // g += lh * conj(v)  ==  conj(conj(lh) * v)
        const double2 gt = conjmul(a.xn[H][p], lh);
        const double2 gc = conjmul(dm, lh);
        a.grad[T0 + H][p] = cadd(a.grad[T0 + H][p], gt);
        a.grad[C0 + H][p] = cadd(a.grad[C0 + H][p], gc);
        if (r.src >= 0) a.grad[r.src][p] = cadd(a.grad[r.src][p], lh);
    }
    a.v[H][p] = conjmul(a.co[C0 + H][p], lh);
    const double2 nl = conjmul(a.co[T0 + H][p], lh);
    a.lam[H][p] = nl;
    if (a.acc[0]) a.acc[H][p] = cadd(a.acc[H][p], nl);
}

// GRAD = false: propagate lam only (no coefficient gradients, x not read).
template <bool GRAD>
__global__ void adjoint_h_kernel(const AdjArgs a) {
    const size_t n = (size_t)a.nx * a.ny * a.nz;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % a.nx), j = (int)((p / a.nx) % a.ny), k = (int)(p / ((size_t)a.nx * a.ny));
        // A_comp for the three H components: contributions of the E splits reading them
        double2 A[3] = {c2(0, 0), c2(0, 0), c2(0, 0)};
        adj_h_term<EXY>(a, p, i, j, k, A);
        adj_h_term<EXZ>(a, p, i, j, k, A);
        adj_h_term<EYX>(a, p, i, j, k, A);
        adj_h_term<EYZ>(a, p, i, j, k, A);
        adj_h_term<EZX>(a, p, i, j, k, A);
        adj_h_term<EZY>(a, p, i, j, k, A);
        adj_h_split<GRAD, HXY>(a, p, i, j, k, A);
        adj_h_split<GRAD, HXZ>(a, p, i, j, k, A);
        adj_h_split<GRAD, HYX>(a, p, i, j, k, A);
        adj_h_split<GRAD, HYZ>(a, p, i, j, k, A);
        adj_h_split<GRAD, HZX>(a, p, i, j, k, A);
        adj_h_split<GRAD, HZY>(a, p, i, j, k, A);
    }
}

// Contribution of H split H to the E components' adjoint: -sign_h D^+_{d(h)} v_h,
// v_h = conj(c_h) lh_h (formed by the H kernel).
template <int H>
__device__ __forceinline__ void adj_e_term(const AdjArgs &a, size_t p, int i, int j, int k, double2 B[3]) {
    constexpr Rule r = rule_of(H);
    constexpr int comp = (r.a - 6) / 2;   // E component read
    const long long q = shifted<r.d, +1>(i, j, k, a);
    const double2 v0 = a.v[H][p];
    const double2 v1 = q < 0 ? c2(0, 0) : a.v[H][q];
    B[comp] = cadd(B[comp], csign<-r.sign>(csub(v1, v0)));
}

template <bool GRAD, int E>
__device__ __forceinline__ void adj_e_split(const AdjArgs &a, size_t p, int i, int j, int k, const double2 B[3]) {
    constexpr Rule r = rule_of(E);
    const double2 mu = a.lam[E][p];
    if (GRAD) {
        const long long q = shifted<r.d, +1>(i, j, k, a);
        const double2 f0 = cadd(a.xn1[r.a][p], a.xn1[r.b][p]);
        const double2 f1 = q < 0 ? c2(0, 0) : cadd(a.xn1[r.a][q], a.xn1[r.b][q]);
        const double2 dp = csign<r.sign>(csub(f1, f0));
        a.grad[T0 + E][p] = cadd(a.grad[T0 + E][p], conjmul(a.xn[E][p], mu));
        a.grad[C0 + E][p] = cadd(a.grad[C0 + E][p], conjmul(dp, mu));
        if (r.src >= 0) a.grad[r.src][p] = cadd(a.grad[r.src][p], mu);
    }
    const double2 nl = cadd(conjmul(a.co[T0 + E][p], mu), B[(E - 6) / 2]);
    a.lam[E][p] = nl;
    a.w[E - 6][p] = conjmul(a.co[C0 + E][p], nl);
    if (a.acc[0]) a.acc[E][p] = cadd(a.acc[E][p], nl);
}

template <bool GRAD>
__global__ void adjoint_e_kernel(const AdjArgs a) {
    const size_t n = (size_t)a.nx * a.ny * a.nz;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % a.nx), j = (int)((p / a.nx) % a.ny), k = (int)(p / ((size_t)a.nx * a.ny));
        // B_comp for the three E components: contributions of the H splits reading them
        double2 B[3] = {c2(0, 0), c2(0, 0), c2(0, 0)};
        adj_e_term<HXY>(a, p, i, j, k, B);
        adj_e_term<HXZ>(a, p, i, j, k, B);
        adj_e_term<HYX>(a, p, i, j, k, B);
        adj_e_term<HYZ>(a, p, i, j, k, B);
        adj_e_term<HZX>(a, p, i, j, k, B);
        adj_e_term<HZY>(a, p, i, j, k, B);
        adj_e_split<GRAD, EXY>(a, p, i, j, k, B);
        adj_e_split<GRAD, EXZ>(a, p, i, j, k, B);
        adj_e_split<GRAD, EYX>(a, p, i, j, k, B);
        adj_e_split<GRAD, EYZ>(a, p, i, j, k, B);
        adj_e_split<GRAD, EZX>(a, p, i, j, k, B);
        adj_e_split<GRAD, EZY>(a, p, i, j, k, B);
    }
}

// w_e = conj(c_e) lam_e for the six E splits: the first H kernel's input.
__global__ void adjoint_w_kernel(const AdjArgs a) {
    const size_t n = (size_t)a.nx * a.ny * a.nz;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
        for (int e = 0; e < 6; ++e) a.w[e][p] = conjmul(a.co[C0 + EXY + e][p], a.lam[EXY + e][p]);
}

// ---- d J / d Re(eps) from the coefficient gradients (chain rule of Eqs. 3-5) ----

struct EpsGradArgs {
    const double2 *eps;
    const double *sig_e;
    const double2 *g[28];
    double *out;
    int nx, ny, nz;
    double omega, tau;
    int k_s;
    double2 hinc;            // incident H_y at k_s (SrcExy = -sign(Exy) c_Exy H_inc = c_Exy H_inc)
};

__device__ __forceinline__ double2 cexpi(double t) { double s, c; sincos(t, &s, &c); return c2(c, s); }

// dJ/deps = Re sum_a conj(G_a) d(coef_a)/d(eps), with sigma held fixed (the
// coefficient gradients G follow the complex-autograd convention 2 dJ/dconj).
__global__ void eps_grad_kernel(const EpsGradArgs a) {
    const size_t n = (size_t)a.nx * a.ny * a.nz, plane = (size_t)a.nx * a.ny;
    const double wt = a.omega * a.tau;
    const double2 e_m1 = cexpi(-wt), e_p1 = cexpi(wt), e_mh = cexpi(-0.5 * wt), e_ph = cexpi(0.5 * wt);
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(p / plane);
        const double eps = a.eps[p].x, sig_mat = a.omega * a.eps[p].y;
        double acc = 0.0;
        for (int e = 6; e < 12; ++e) {
            const double sg = sig_mat + ((e == EXY || e == EYX) ? a.sig_e[k] : 0.0);   // z-difference splits
            double2 dt, dc;
            if (eps > 0.0) {
                const double den = 1.0 + a.tau * sg / eps;
                dt = cscale((a.tau * sg / (eps * eps)) / (den * den), e_m1);
                const double den2 = eps + a.tau * sg;
                dc = cscale(-a.tau / (den2 * den2), e_mh);
            } else {
                const double den = 1.0 - a.tau * sg / eps;
                dt = cscale(-(a.tau * sg / (eps * eps)) / (den * den), e_p1);
                const double den2 = eps - a.tau * sg;
                dc = cscale(a.tau / (den2 * den2), e_ph);
            }
            acc += conjmul(a.g[T0 + e][p], dt).x + conjmul(a.g[C0 + e][p], dc).x;
            if (e == EXY && k == a.k_s) {
                const double2 ds = c2(dc.x * a.hinc.x - dc.y * a.hinc.y, dc.x * a.hinc.y + dc.y * a.hinc.x);
                acc += conjmul(a.g[SRC_EXY][p], ds).x;
            }
        }
        a.out[p] = acc;
    }
}

int ensure_adjoint_scratch(thiim_ctx *c, int n_back) {
    if (!c->adj_lh[0]) {
        for (int i = 0; i < 6; ++i)
            if (cudaMalloc(&c->adj_lh[i], c->n_cells * 16) != cudaSuccess) { cudaGetLastError(); return THIIM_ERR_NOMEM; }
    }
    if (!c->adj_w[0]) {
        for (int i = 0; i < 6; ++i)
            if (cudaMalloc(&c->adj_w[i], c->n_cells * 16) != cudaSuccess) { cudaGetLastError(); return THIIM_ERR_NOMEM; }
    }
    if (c->adj_cap < n_back) {
        for (int m = 0; m < c->adj_cap; ++m)
            for (int i = 0; i < THIIM_N_FIELDS; ++i) { cudaFree(c->adj_states[m][i]); c->adj_states[m][i] = nullptr; }
        c->adj_cap = 0;
        for (int m = 0; m < n_back; ++m)
            for (int i = 0; i < THIIM_N_FIELDS; ++i)
                if (cudaMalloc(&c->adj_states[m][i], c->n_cells * 16) != cudaSuccess) {
                    cudaGetLastError();
                    c->adj_cap = m;   // states 0..m-1 complete; the partial one is freed at destroy
                    return THIIM_ERR_NOMEM;
                }
        c->adj_cap = n_back;
    }
    return THIIM_OK;
}

}  // namespace

extern "C" int thiim_adjoint_iterate(thiim_ctx *c, void *const lambda[THIIM_N_FIELDS],
                                     void *const grad_coeff[THIIM_N_COEFFS],
                                     const void *const fwd_checkpoint[THIIM_N_FIELDS], int n_back) {
    if (!c || !lambda || !grad_coeff || !fwd_checkpoint || n_back < 1 || n_back > THIIM_MAX_ADJOINT_SEGMENT)
        return THIIM_ERR_ARG;
    if (c->precision != THIIM_C128) return THIIM_ERR_ARG;
    if (!c->have_coeffs || c->use_table) return THIIM_ERR_STATE;
    for (int i = 0; i < THIIM_N_FIELDS; ++i)
        if (!lambda[i] || !fwd_checkpoint[i] || !aligned(lambda[i], 16) || !aligned(fwd_checkpoint[i], 16))
            return lambda[i] && fwd_checkpoint[i] ? THIIM_ERR_ALIGN : THIIM_ERR_ARG;
    for (int i = 0; i < THIIM_N_COEFFS; ++i)
        if (!grad_coeff[i] || !aligned(grad_coeff[i], 16)) return grad_coeff[i] ? THIIM_ERR_ALIGN : THIIM_ERR_ARG;
    int st = ensure_adjoint_scratch(c, n_back);
    if (st) return st;

    // Recompute x^{n0+1} .. x^{n0+n_back} from the checkpoint x^{n0}.
    const int tx = tiles_x(c), ty = tiles_y(c);
    const int chunks = (c->nz + c->zchunk - 1) / c->zchunk;
    const dim3 grid((unsigned)(tx * ty), (unsigned)chunks);
    SweepArgs s;
    memset(&s, 0, sizeof(s));
    memcpy(s.co, c->coeff, sizeof(s.co));
    s.nx = c->nx; s.ny = c->ny; s.nz = c->nz;
    s.bc = c->bc;
    s.zchunk = c->zchunk;
    s.tiles_x = tx;
    for (int m = 0; m < n_back; ++m) {
        for (int i = 0; i < THIIM_N_FIELDS; ++i) {
            s.src[i] = m == 0 ? fwd_checkpoint[i] : c->adj_states[m - 1][i];
            s.dst[i] = c->adj_states[m][i];
        }
        if (launch_sweep_f64_ctx(c, s, grid) != cudaSuccess) return THIIM_ERR_CUDA;
    }
    // Reverse steps n0+n_back-1 .. n0.
    AdjArgs a;
    memset(&a, 0, sizeof(a));
    for (int i = 0; i < THIIM_N_FIELDS; ++i) a.lam[i] = (double2 *)lambda[i];
    for (int i = 0; i < THIIM_N_COEFFS; ++i) {
        a.grad[i] = (double2 *)grad_coeff[i];
        a.co[i] = (const double2 *)c->coeff[i];
    }
    for (int i = 0; i < 6; ++i) {
        a.v[i] = (double2 *)c->adj_lh[i];
        a.w[i] = (double2 *)c->adj_w[i];
    }
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
    a.bc = c->bc;
    size_t blocks = (c->n_cells + 255) / 256;
    if (blocks > 8u * (size_t)c->num_sms) blocks = 8u * (size_t)c->num_sms;
    adjoint_w_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(a);
    for (int m = n_back - 1; m >= 0; --m) {
        for (int i = 0; i < THIIM_N_FIELDS; ++i) {
            a.xn[i] = (const double2 *)(m == 0 ? fwd_checkpoint[i] : c->adj_states[m - 1][i]);
            a.xn1[i] = (const double2 *)c->adj_states[m][i];
        }
        adjoint_h_kernel<true><<<(unsigned)blocks, 256, 0, c->stream>>>(a);
        adjoint_e_kernel<true><<<(unsigned)blocks, 256, 0, c->stream>>>(a);
        if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
    }
    return THIIM_OK;
}

namespace {

struct NormArgs {
    const double2 *w[12];
    const double2 *s[12];
    size_t n;
    double *partials;
};

// Per-CTA |w|^2 and |s|^2 over the 12 arrays (fixed-order reductions).
__global__ void __launch_bounds__(256) adj_norm_kernel(const NormArgs a) {
    __shared__ double rw[8], rs[8];
    double aw = 0.0, as = 0.0;
    for (size_t p = (size_t)blockIdx.x * 256 + threadIdx.x; p < a.n; p += (size_t)gridDim.x * 256) {
        for (int i = 0; i < 12; ++i) {
            const double2 u = a.w[i][p], v = a.s[i][p];
            aw += u.x * u.x + u.y * u.y;
            as += v.x * v.x + v.y * v.y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        aw += __shfl_down_sync(0xffffffffu, aw, o);
        as += __shfl_down_sync(0xffffffffu, as, o);
    }
    if ((threadIdx.x & 31) == 0) { rw[threadIdx.x >> 5] = aw; rs[threadIdx.x >> 5] = as; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tw = 0.0, ts = 0.0;
        for (int i = 0; i < 8; ++i) { tw += rw[i]; ts += rs[i]; }
        a.partials[2 * blockIdx.x] = tw;
        a.partials[2 * blockIdx.x + 1] = ts;
    }
}

// |last term| / |sum| on the host (synchronises the stream).
int adj_rel(thiim_ctx *c, void *const *w, void *const *s, double *rel) {
    const size_t ctas = 4 * (size_t)c->num_sms;
    int st = ensure_partials(c, ctas);
    if (st) return st;
    if (!c->adj_norms && cudaMalloc(&c->adj_norms, 2 * sizeof(double)) != cudaSuccess) return THIIM_ERR_NOMEM;
    NormArgs a;
    for (int i = 0; i < 12; ++i) { a.w[i] = (const double2 *)w[i]; a.s[i] = (const double2 *)s[i]; }
    a.n = c->n_cells;
    a.partials = c->partials;
    adj_norm_kernel<<<(unsigned)ctas, 256, 0, c->stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
    if (finalize_norms(c->partials, ctas, c->adj_norms, c->stream) != cudaSuccess) return THIIM_ERR_CUDA;
    double h[2];
    if (cudaMemcpyAsync(h, c->adj_norms, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return THIIM_ERR_CUDA;
    if (!isfinite(h[0]) || !isfinite(h[1])) return THIIM_ERR_NONFINITE;
    *rel = h[1] > 0.0 ? sqrt(h[0] / h[1]) : 0.0;
    return THIIM_OK;
}

}  // namespace

extern "C" int thiim_adjoint_steady(thiim_ctx *c, void *const lambda[THIIM_N_FIELDS],
                                    void *const grad_coeff[THIIM_N_COEFFS],
                                    const void *const x_star[THIIM_N_FIELDS], int max_iters, int check_every,
                                    double tol, int *iters_out, double *rel_out) {
    if (!c || !lambda || !grad_coeff || !x_star || max_iters < 1 || check_every < 1 || !(tol >= 0.0) ||
        !isfinite(tol))
        return THIIM_ERR_ARG;
    if (c->precision != THIIM_C128) return THIIM_ERR_ARG;
    if (!c->have_coeffs || c->use_table) return THIIM_ERR_STATE;
    for (int i = 0; i < THIIM_N_FIELDS; ++i)
        if (!lambda[i] || !x_star[i] || !aligned(lambda[i], 16) || !aligned(x_star[i], 16))
            return lambda[i] && x_star[i] ? THIIM_ERR_ALIGN : THIIM_ERR_ARG;
    for (int i = 0; i < THIIM_N_COEFFS; ++i)
        if (!grad_coeff[i] || !aligned(grad_coeff[i], 16)) return grad_coeff[i] ? THIIM_ERR_ALIGN : THIIM_ERR_ARG;
    int st = ensure_adjoint_scratch(c, 1);
    if (st) return st;
    void **w = c->adj_states[0];     // the current term (M^H)^k g
    const size_t bytes = c->n_cells * 16;
    for (int i = 0; i < THIIM_N_FIELDS; ++i)
        if (cudaMemcpyAsync(w[i], lambda[i], bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            return THIIM_ERR_CUDA;
    AdjArgs a;
    memset(&a, 0, sizeof(a));
    for (int i = 0; i < THIIM_N_FIELDS; ++i) {
        a.lam[i] = (double2 *)w[i];
        a.acc[i] = (double2 *)lambda[i];          // lam* so far (starts as g)
    }
    for (int i = 0; i < THIIM_N_COEFFS; ++i) a.co[i] = (const double2 *)c->coeff[i];
    for (int i = 0; i < 6; ++i) {
        a.v[i] = (double2 *)c->adj_lh[i];
        a.w[i] = (double2 *)c->adj_w[i];
    }
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
    a.bc = c->bc;
    size_t blocks = (c->n_cells + 255) / 256;
    if (blocks > 8u * (size_t)c->num_sms) blocks = 8u * (size_t)c->num_sms;
    adjoint_w_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(a);
    int k = 1;
    double rel = 1.0;
    bool have_rel = false;
    while (k < max_iters) {
        adjoint_h_kernel<false><<<(unsigned)blocks, 256, 0, c->stream>>>(a);
        adjoint_e_kernel<false><<<(unsigned)blocks, 256, 0, c->stream>>>(a);
        if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
        ++k;
        have_rel = false;
        if (tol > 0.0 && (k % check_every == 0)) {
            st = adj_rel(c, w, lambda, &rel);
            if (st) return st;
            have_rel = true;
            if (rel <= tol) break;
        }
    }
    if (!have_rel) {
        st = adj_rel(c, w, lambda, &rel);
        if (st) return st;
    }
    // Gradient of lam*: the gradient kernels on a copy (they overwrite their lam).
    for (int i = 0; i < THIIM_N_FIELDS; ++i)
        if (cudaMemcpyAsync(w[i], lambda[i], bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            return THIIM_ERR_CUDA;
    for (int i = 0; i < THIIM_N_FIELDS; ++i) {
        a.acc[i] = nullptr;
        a.xn[i] = (const double2 *)x_star[i];
        a.xn1[i] = (const double2 *)x_star[i];
    }
    for (int i = 0; i < THIIM_N_COEFFS; ++i) a.grad[i] = (double2 *)grad_coeff[i];
    adjoint_w_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(a);
    adjoint_h_kernel<true><<<(unsigned)blocks, 256, 0, c->stream>>>(a);
    adjoint_e_kernel<true><<<(unsigned)blocks, 256, 0, c->stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
    if (iters_out) *iters_out = k;
    if (rel_out) *rel_out = rel;
    return THIIM_OK;
}

extern "C" int thiim_build_coeffs_grad(thiim_ctx *c, const void *eps_r, const double *sigma_pml_e, double omega,
                                       double tau, int k_s, double amp_re, double amp_im,
                                       const void *const grad_coeff[THIIM_N_COEFFS], double *grad_eps_re) {
    if (!c || !eps_r || !grad_coeff || !grad_eps_re || !(tau > 0.0) || k_s >= c->nz) return THIIM_ERR_ARG;
    if (!aligned(eps_r, 16) || !aligned(grad_eps_re, 8)) return THIIM_ERR_ALIGN;
    for (int i = 0; i < THIIM_N_COEFFS; ++i)
        if (!grad_coeff[i] || !aligned(grad_coeff[i], 16)) return grad_coeff[i] ? THIIM_ERR_ALIGN : THIIM_ERR_ARG;
    const double wt = 2.0 * sin(0.5 * omega * tau) / tau;
    if (k_s >= 0 && !(fabs(wt) <= 2.0 && wt != 0.0)) return THIIM_ERR_ARG;
    if (!c->pml) {
        if (cudaMalloc(&c->pml, 2 * (size_t)c->nz * sizeof(double)) != cudaSuccess) return THIIM_ERR_NOMEM;
        if (cudaMalloc(&c->flag, sizeof(int)) != cudaSuccess) return THIIM_ERR_NOMEM;
    }
    if (sigma_pml_e) {
        if (cudaMemcpyAsync(c->pml, sigma_pml_e, (size_t)c->nz * sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return THIIM_ERR_CUDA;
    } else if (cudaMemsetAsync(c->pml, 0, (size_t)c->nz * sizeof(double), c->stream) != cudaSuccess) {
        return THIIM_ERR_CUDA;
    }
    EpsGradArgs a;
    memset(&a, 0, sizeof(a));
    a.eps = (const double2 *)eps_r;
    a.sig_e = c->pml;
    for (int i = 0; i < THIIM_N_COEFFS; ++i) a.g[i] = (const double2 *)grad_coeff[i];
    a.out = grad_eps_re;
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
    a.omega = omega; a.tau = tau;
    a.k_s = k_s;
    if (k_s >= 0) {   // H_inc(k_s) = -amp (1 - e^{i kappa}) / (i omega_t)
        const double kappa = 2.0 * asin(0.5 * wt);
        const double dre = 1.0 - cos(kappa), dim = -sin(kappa);
        const double nre = -(amp_re * dre - amp_im * dim), nim = -(amp_re * dim + amp_im * dre);
        a.hinc = make_double2(nim / wt, -nre / wt);
    }
    size_t blocks = (c->n_cells + 255) / 256;
    if (blocks > 8u * (size_t)c->num_sms) blocks = 8u * (size_t)c->num_sms;
    eps_grad_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? THIIM_OK : THIIM_ERR_CUDA;
}
