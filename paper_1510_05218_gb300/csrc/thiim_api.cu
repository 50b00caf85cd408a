// C ABI of the THIIM sweep library: context, argument checks, launches,
// the residual reduction and the coefficient builder.  See include/thiim.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "../../include/thiim.h"
#include "thiim_ctx.h"

using namespace thiim;

namespace thiim {

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Tile shape by precision (matches Tile<A> of the kernels the precision runs).
int tile_w(const thiim_ctx *c) {
    return c->precision == THIIM_C128_PAIR ? Tile<PairArith<1, 1>>::TX
         : c->precision == THIIM_C128      ? Tile<Native<double>>::TX : Tile<Native<float>>::TX;
}
int tile_h(const thiim_ctx *c) {
    if (c->precision == THIIM_C128)   // the tall FP64 tile on large grids
        return c->n_cells >= THIIM_F64_TALL_MIN_CELLS ? Tile<Native<double>>::TY : SWEEP_TY;
    return c->precision == THIIM_C128_PAIR ? Tile<PairArith<1, 1>>::TY : Tile<Native<float>>::TY;
}

cudaError_t launch_sweep_f64_ctx(const thiim_ctx *c, const SweepArgs &a, dim3 grid) {
    return tile_h(c) == SWEEP_TY ? launch_sweep_f64_t8(a, grid, c->stream) : launch_sweep_f64(a, grid, c->stream);
}
int tiles_x(const thiim_ctx *c) { return (c->nx + tile_w(c) - 1) / tile_w(c); }
int tiles_y(const thiim_ctx *c) { return (c->ny + tile_h(c) - 1) / tile_h(c); }

// Planes per CTA: enough CTAs along z that the grid covers every SM several
// times, but at least 8 planes so the one-plane prologue and lookahead of a
// chunk stay cheap.
int default_zchunk(const thiim_ctx *c) {
    const long tiles = (long)tiles_x(c) * tiles_y(c);
    const long target = 8L * c->num_sms;
    long chunks = (target + tiles - 1) / tiles;
    long maxchunks = c->nz / 8 > 0 ? c->nz / 8 : 1;
    if (chunks > maxchunks) chunks = maxchunks;
    if (chunks < 1) chunks = 1;
    return (int)((c->nz + chunks - 1) / chunks);
}

int ensure_partials(thiim_ctx *c, size_t ctas) {
    if (c->partials_cap >= ctas) return THIIM_OK;
    if (c->partials) cudaFree(c->partials);
    c->partials = nullptr;
    c->partials_cap = 0;
    if (cudaMalloc(&c->partials, 2 * ctas * sizeof(double)) != cudaSuccess) return THIIM_ERR_NOMEM;
    c->partials_cap = ctas;
    return THIIM_OK;
}

// Sum the per-CTA partial pairs in a fixed order (deterministic).
__global__ void finalize_norms_kernel(const double *partials, size_t n, double *out) {
    __shared__ double sd[256], sx[256];
    double d = 0.0, x = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        d += partials[2 * i];
        x += partials[2 * i + 1];
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
    if (threadIdx.x == 0) { out[0] = sd[0]; out[1] = sx[0]; }
}

cudaError_t finalize_norms(const double *partials, size_t n, double *out, cudaStream_t s) {
    finalize_norms_kernel<<<1, 256, 0, s>>>(partials, n, out);
    return cudaGetLastError();
}

}  // namespace thiim

namespace {

// ---- coefficient builder (Eqs. 3-5 solved for the new value) ---------------

struct dc { double x, y; };
__device__ __forceinline__ dc mk(double x, double y) { dc r; r.x = x; r.y = y; return r; }
__device__ __forceinline__ dc cmul(dc a, dc b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ dc cdiv(dc a, dc b) {
    const double den = b.x * b.x + b.y * b.y;
    return mk((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ dc cexpi(double t) { double s, c; sincos(t, &s, &c); return mk(c, s); }

struct BuildArgs {
    const double2 *eps;
    const double *sig_e;      // nz
    const double *sig_h;      // nz
    void *co[THIIM_N_COEFFS];
    int nx, ny, nz;
    double omega, tau;
    int k_s;                  // -1: no source
    dc src_h;                 // factor of c_Hyx at k_s (x polarisation)
    dc src_e;                 // factor of c_Exy at k_s
    bool pol_y;               // the wave has a y component:
    dc src_hxy;               // factor of c_Hxy at k_s
    dc src_eyx;               // factor of c_Eyx at k_s
    int *flag;
};

// Splits that difference along z carry the absorbing-layer conductivity.
__device__ __forceinline__ bool along_z(int s) { return s == HXY || s == HYX || s == EXY || s == EYX; }

template <typename V>
__device__ __forceinline__ void put(void *base, size_t i, dc v) {
    V w;
    w.x = (decltype(w.x))v.x;
    w.y = (decltype(w.y))v.y;
    reinterpret_cast<V *>(base)[i] = w;
}

// The 28 coefficients of one cell: material eps (real part) and conductivity
// sigma_mat = omega Im(eps_r), absorbing-layer conductivities of its planes.
__device__ __forceinline__ void cell_coeffs(const BuildArgs &a, double eps, double sig_mat, int k, dc out[28]) {
    const double wt = a.omega * a.tau;
    const dc e_mh = cexpi(-0.5 * wt), e_ph = cexpi(0.5 * wt);
    const dc e_m1 = cexpi(-wt), e_p1 = cexpi(wt);
    for (int s = 0; s < 12; ++s) {
        dc t, c;
        if (s < 6) {             // H, Eq. 4 (mu = 1)
            const double ss = along_z(s) ? a.sig_h[k] : 0.0;
            const dc den = mk(e_ph.x + a.tau * ss, e_ph.y);
            t = cdiv(e_mh, den);
            c = cdiv(mk(a.tau, 0.0), den);
        } else {
            const double sg = sig_mat + (along_z(s) ? a.sig_e[k] : 0.0);
            if (eps > 0.0) {     // Eq. 3
                t = cdiv(e_m1, mk(1.0 + a.tau * sg / eps, 0.0));
                c = cdiv(mk(a.tau * e_mh.x, a.tau * e_mh.y), mk(eps + a.tau * sg, 0.0));
            } else {             // Eq. 5, back iteration
                t = cdiv(e_p1, mk(1.0 - a.tau * sg / eps, 0.0));
                c = cdiv(mk(-a.tau * e_ph.x, -a.tau * e_ph.y), mk(eps - a.tau * sg, 0.0));
            }
        }
        out[T0 + s] = t;
        out[C0 + s] = c;
    }
    out[SRC_HXY] = (a.pol_y && k == a.k_s) ? cmul(out[C0 + HXY], a.src_hxy) : mk(0, 0);
    out[SRC_EYX] = (a.pol_y && k == a.k_s) ? cmul(out[C0 + EYX], a.src_eyx) : mk(0, 0);
    out[SRC_HYX] = k == a.k_s ? cmul(out[C0 + HYX], a.src_h) : mk(0, 0);
    out[SRC_EXY] = k == a.k_s ? cmul(out[C0 + EXY], a.src_e) : mk(0, 0);
}

template <typename V>
__global__ void build_coeffs_kernel(const BuildArgs a) {
    const size_t n = (size_t)a.nx * a.ny * a.nz;
    const size_t plane = (size_t)a.nx * a.ny;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(p / plane);
        const double2 er = a.eps[p];
        if (!(er.x != 0.0) || !isfinite(er.x) || !isfinite(er.y)) atomicOr(a.flag, 1);
        dc v[28];
        cell_coeffs(a, er.x, a.omega * er.y, k, v);
        for (int i = 0; i < 28; ++i) put<V>(a.co[i], p, v[i]);
    }
}

// Table of the compressed variant: row (m, k) holds the 28 coefficients of a
// cell of material m on plane k.  a.eps holds the n_mat permittivities.
template <typename V>
__global__ void build_table_kernel(const BuildArgs a, int n_mat, void *table) {
    const int rows = n_mat * a.nz;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        const int m = r / a.nz, k = r % a.nz;
        const double2 er = a.eps[m];
        if (!(er.x != 0.0) || !isfinite(er.x) || !isfinite(er.y)) atomicOr(a.flag, 1);
        dc v[28];
        cell_coeffs(a, er.x, a.omega * er.y, k, v);
        for (int i = 0; i < 28; ++i) put<V>(table, (size_t)r * 28 + i, v[i]);
    }
}

// Checks the builder's scalar arguments, uploads the absorbing-layer
// conductivities and fills the scalar part of the builder's arguments.
int prepare_build(thiim_ctx *c, const double *sigma_pml_e, const double *sigma_pml_h, double omega, double tau,
                  int k_s, const double jones[4], BuildArgs *out) {
    if (!(tau > 0.0) || !isfinite(omega) || !isfinite(tau) || k_s >= c->nz) return THIIM_ERR_ARG;
    for (int i = 0; i < 4; ++i)
        if (!isfinite(jones[i])) return THIIM_ERR_ARG;
    // Discrete frequency of the fixed point and the incident wave number:
    // omega_t = 2 sin(omega tau / 2) / tau, 2 sin(kappa / 2) = omega_t.
    const double wt = 2.0 * sin(0.5 * omega * tau) / tau;
    if (k_s >= 0 && !(fabs(wt) <= 2.0)) return THIIM_ERR_ARG;
    if (!c->pml) {
        if (cudaMalloc(&c->pml, 2 * (size_t)c->nz * sizeof(double)) != cudaSuccess) return THIIM_ERR_NOMEM;
        if (cudaMalloc(&c->flag, sizeof(int)) != cudaSuccess) return THIIM_ERR_NOMEM;
    }
    double *host = (double *)calloc(2 * (size_t)c->nz, sizeof(double));
    if (!host) return THIIM_ERR_NOMEM;
    if (sigma_pml_e) memcpy(host, sigma_pml_e, (size_t)c->nz * sizeof(double));
    if (sigma_pml_h) memcpy(host + c->nz, sigma_pml_h, (size_t)c->nz * sizeof(double));
    cudaError_t e = cudaMemcpyAsync(c->pml, host, 2 * (size_t)c->nz * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // host buffer may go away
    free(host);
    if (e != cudaSuccess) return THIIM_ERR_CUDA;

    BuildArgs &a = *out;
    memset(&a, 0, sizeof(a));
    a.sig_e = c->pml;
    a.sig_h = c->pml + c->nz;
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
    a.omega = omega; a.tau = tau;
    a.k_s = k_s;
    a.flag = c->flag;
    if (k_s >= 0) {
        // Hyx (sign -1) at the scattered-field H plane k_s reads the incident
        // E_x(k_s) = A_x:  Src = +c_Hyx * A_x.
        // Exy (sign -1) at the total-field E plane k_s reads the incident
        // H_y(k_s) = -(E_inc(k_s) - E_inc(k_s - 1)) / (i omega_t)
        //          = -A_x (1 - e^{i kappa}) / (i omega_t):  Src = +c_Exy * H_y.
        // The y component (E_y, H_x = +dE_y / (i omega_t)) enters through
        // Hxy and Eyx (sign +1):  Src = -c_Hxy * A_y, Src = -c_Eyx * H_x.
        const double kappa = 2.0 * asin(0.5 * wt);
        const double dre = 1.0 - cos(kappa), dim = -sin(kappa);   // 1 - e^{i kappa}
        // -A (1 - e^{i kappa}) / (i omega_t); (n_re + i n_im) / (i wt) = (n_im - i n_re) / wt
        auto h_factor = [&](double are, double aim, dc *f) {
            const double nre = -(are * dre - aim * dim), nim = -(are * dim + aim * dre);
            f->x = nim / wt; f->y = -nre / wt;
        };
        a.src_h.x = jones[0]; a.src_h.y = jones[1];
        h_factor(jones[0], jones[1], &a.src_e);
        a.pol_y = jones[2] != 0.0 || jones[3] != 0.0;
        a.src_hxy.x = -jones[2]; a.src_hxy.y = -jones[3];
        h_factor(jones[2], jones[3], &a.src_eyx);   // -H_x = -A_y (1 - e^{i kappa}) / (i omega_t)
    }
    return THIIM_OK;
}

// Waits for the builder and reports a zero or non-finite permittivity.
int read_build_flag(thiim_ctx *c) {
    int flag = 0;
    if (cudaMemcpyAsync(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return THIIM_ERR_CUDA;
    return flag ? THIIM_ERR_ARG : THIIM_OK;
}

}  // namespace

extern "C" {

int thiim_version(void) { return 1 * 10000 + 0 * 100 + 0; }

const char *thiim_strerror(int status) {
    switch (status) {
        case THIIM_OK: return "ok";
        case THIIM_ERR_ARG: return "invalid argument";
        case THIIM_ERR_ALIGN: return "misaligned array";
        case THIIM_ERR_STATE: return "call order violated (fields or coefficients not set, or no iteration yet)";
        case THIIM_ERR_CUDA: return "CUDA runtime error";
        case THIIM_ERR_TIMEOUT: return "bounded device wait expired";
        case THIIM_ERR_NONFINITE: return "non-finite value in a reduction";
        case THIIM_ERR_NOMEM: return "device allocation failed";
        default: return "unknown status";
    }
}

int thiim_create(thiim_ctx **out, int nx, int ny, int nz, int precision, unsigned bc_flags,
                 void *cuda_stream) {
    if (!out) return THIIM_ERR_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return THIIM_ERR_ARG;
    if ((double)nx * ny * nz > (double)(1ull << 40)) return THIIM_ERR_ARG;
    if (precision != THIIM_C128 && precision != THIIM_C64 && precision != THIIM_C128_PAIR) return THIIM_ERR_ARG;
    if (bc_flags & ~7u) return THIIM_ERR_ARG;
    thiim_ctx *c = new (std::nothrow) thiim_ctx();
    if (!c) return THIIM_ERR_NOMEM;
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->precision = precision;
    c->bc = bc_flags;
    c->stream = (cudaStream_t)cuda_stream;
    c->elem = precision == THIIM_C64 ? 8 : 16;
    c->n_cells = (size_t)nx * ny * nz;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return THIIM_ERR_CUDA;
    }
    c->zchunk = default_zchunk(c);
    c->temporal = 1;
    c->fp64_int_ops = precision == THIIM_C128 ? THIIM_FP64_INT_OPS_DEFAULT : 0u;
    *out = c;
    return THIIM_OK;
}

int thiim_set_tuning(thiim_ctx *c, int temporal_block, int zchunk) {
    if (!c || zchunk < 0 || zchunk > c->nz) return THIIM_ERR_ARG;
    if (temporal_block != 1 && temporal_block != 2) return THIIM_ERR_ARG;
    if (temporal_block == 2 && c->precision != THIIM_C64) return THIIM_ERR_ARG;
    c->temporal = temporal_block;
    c->zchunk = zchunk ? zchunk : default_zchunk(c);
    return THIIM_OK;
}

int thiim_set_fp64_int_ops(thiim_ctx *c, unsigned ops) {
    if (!c || c->precision != THIIM_C128) return THIIM_ERR_ARG;
    if (ops != 0u && ops != THIIM_INT_ADD && ops != (THIIM_INT_ADD | THIIM_INT_MUL) && ops != THIIM_INT_SUMS)
        return THIIM_ERR_ARG;
    c->fp64_int_ops = ops;
    return THIIM_OK;
}

int thiim_set_stream(thiim_ctx *c, void *cuda_stream) {
    if (!c) return THIIM_ERR_ARG;
    c->stream = (cudaStream_t)cuda_stream;
    return THIIM_OK;
}

int thiim_set_coeffs(thiim_ctx *c, void *const coeff[THIIM_N_COEFFS]) {
    if (!c || !coeff) return THIIM_ERR_ARG;
    for (int i = 0; i < THIIM_N_COEFFS; ++i) {
        if (!coeff[i]) return THIIM_ERR_ARG;
        if (!aligned(coeff[i], c->elem)) return THIIM_ERR_ALIGN;
    }
    memcpy(c->coeff, coeff, sizeof(c->coeff));
    c->have_coeffs = true;
    c->use_table = false;
    c->pair_dirty = true;
    return THIIM_OK;
}

int thiim_set_material_coeffs(thiim_ctx *c, const unsigned char *mat, int n_mat, const void *table) {
    if (!c || !mat || !table || n_mat < 1 || n_mat > THIIM_MAX_MATERIALS) return THIIM_ERR_ARG;
    if (!aligned(table, c->elem)) return THIIM_ERR_ALIGN;
    c->mat = mat;
    c->table = table;
    c->n_mat = n_mat;
    c->use_table = true;
    c->have_coeffs = true;
    c->pair_table_dirty = true;
    return THIIM_OK;
}

int thiim_set_fields(thiim_ctx *c, void *const field[THIIM_N_FIELDS]) {
    if (!c || !field) return THIIM_ERR_ARG;
    for (int i = 0; i < THIIM_N_FIELDS; ++i) {
        if (!field[i]) return THIIM_ERR_ARG;
        if (!aligned(field[i], c->elem)) return THIIM_ERR_ALIGN;
    }
    if (!c->alt[0]) {
        for (int i = 0; i < THIIM_N_FIELDS; ++i) {
            if (cudaMalloc(&c->alt[i], c->n_cells * c->elem) != cudaSuccess) {
                for (int j = 0; j < i; ++j) { cudaFree(c->alt[j]); c->alt[j] = nullptr; }
                c->alt[i] = nullptr;
                cudaGetLastError();
                return THIIM_ERR_NOMEM;
            }
        }
    }
    memcpy(c->user, field, sizeof(c->user));
    c->have_fields = true;
    c->have_norm = false;
    return THIIM_OK;
}

int thiim_iterate(thiim_ctx *c, int n_iters) {
    if (!c || n_iters < 0) return THIIM_ERR_ARG;
    if (!c->have_fields || !c->have_coeffs) return THIIM_ERR_STATE;
    if (n_iters == 0) return THIIM_OK;
    const int tx = tiles_x(c), ty = tiles_y(c);
    const int chunks = (c->nz + c->zchunk - 1) / c->zchunk;
    // one CTA per (tile, z chunk): the launch's grid limits (x < 2^31, y <= 65535)
    if ((long long)tx * ty > 0x7FFFFFFFLL || chunks > 65535) return THIIM_ERR_ARG;
    const dim3 grid((unsigned)(tx * ty), (unsigned)chunks);
    const size_t ctas = (size_t)tx * ty * chunks;
    // the two-iteration kernel's tiles may be taller
    const int ty2 = (c->ny + SWEEP2_TY - 1) / SWEEP2_TY;
    const dim3 grid2((unsigned)(tx * ty2), (unsigned)chunks);
    const size_t ctas2 = (size_t)tx * ty2 * chunks;
    int st = ensure_partials(c, ctas > ctas2 ? ctas : ctas2);
    if (st) return st;
    if (!c->norms && cudaMalloc(&c->norms, 2 * sizeof(double)) != cudaSuccess) return THIIM_ERR_NOMEM;

    const bool pair = c->precision == THIIM_C128_PAIR;
    const bool tbl = c->use_table;
    if (pair && tbl) {
        const size_t n = (size_t)c->n_mat * c->nz * THIIM_N_COEFFS;
        if (c->pair_table_cap < n) {
            if (c->pair_table) cudaFree(c->pair_table);
            c->pair_table = nullptr;
            c->pair_table_cap = 0;
            if (cudaMalloc(&c->pair_table, n * 16) != cudaSuccess) {
                cudaGetLastError();
                return THIIM_ERR_NOMEM;
            }
            c->pair_table_cap = n;
            c->pair_table_dirty = true;
        }
        if (c->pair_table_dirty) {
            const void *src = c->table;
            void *dst = c->pair_table;
            if (split_coeffs(&src, &dst, 1, n, c->stream) != cudaSuccess) return THIIM_ERR_CUDA;
            c->pair_table_dirty = false;
        }
    } else if (pair) {
        if (!c->pair_co[0]) {
            for (int i = 0; i < THIIM_N_COEFFS; ++i) {
                if (cudaMalloc(&c->pair_co[i], c->n_cells * 16) != cudaSuccess) {
                    for (int j = 0; j < i; ++j) { cudaFree(c->pair_co[j]); c->pair_co[j] = nullptr; }
                    c->pair_co[i] = nullptr;
                    cudaGetLastError();
                    return THIIM_ERR_NOMEM;
                }
            }
            c->pair_dirty = true;
        }
        if (c->pair_dirty) {
            if (split_coeffs(c->coeff, c->pair_co, THIIM_N_COEFFS, c->n_cells, c->stream) != cudaSuccess)
                return THIIM_ERR_CUDA;
            c->pair_dirty = false;
        }
    }

    SweepArgs a;
    memset(&a, 0, sizeof(a));
    memcpy(a.co, pair ? c->pair_co : c->coeff, sizeof(a.co));
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
    a.bc = c->bc;
    a.zchunk = c->zchunk;
    a.tiles_x = tx;
    if (tbl) {
        a.mat = c->mat;
        a.table = pair ? c->pair_table : c->table;
    }
    void **from = c->user, **to = c->alt;
    size_t last_ctas = ctas;     // CTAs (partials) of the last launch
    for (int it = 0; it < n_iters;) {
        // temporal blocking: two iterations per launch while two remain
        // (array coefficients only; the table variant runs one per launch)
        const int step = (c->temporal == 2 && !tbl && n_iters - it >= 2) ? 2 : 1;
        memcpy(a.src, from, sizeof(a.src));
        memcpy(a.dst, to, sizeof(a.dst));
        a.partials = (it + step == n_iters) ? c->partials : nullptr;
        cudaError_t e;
        if (tbl && pair)
            e = launch_sweep_pair_tbl(a, grid, c->stream, it > 0, it < n_iters - 1);
        else if (tbl && c->precision == THIIM_C128)
            e = launch_sweep_f64_tbl(a, grid, c->stream, tile_h(c) != SWEEP_TY);
        else if (tbl)
            e = launch_sweep_f32_tbl(a, grid, c->stream);
        else if (pair)   // intermediate iterates stay as float4 pairs; first reads and last writes complex128
            e = launch_sweep_pair(a, grid, c->stream, it > 0, it < n_iters - 1);
        else if (c->precision == THIIM_C128 && c->fp64_int_ops)
            e = launch_sweep_f64_int(a, grid, c->stream, (int)c->fp64_int_ops, tile_h(c) != SWEEP_TY);
        else if (c->precision == THIIM_C128)
            e = launch_sweep_f64_ctx(c, a, grid);
        else if (step == 2)
            e = launch_sweep2_f32(a, grid2, c->stream);
        else
            e = launch_sweep_f32(a, grid, c->stream);
        if (e != cudaSuccess) return THIIM_ERR_CUDA;
        last_ctas = step == 2 ? ctas2 : ctas;
        void **tmp = from; from = to; to = tmp;
        it += step;
    }
    if (from != c->user) {       // odd count: the newest iterate sits in the library's set
        for (int i = 0; i < THIIM_N_FIELDS; ++i) {
            if (cudaMemcpyAsync(c->user[i], c->alt[i], c->n_cells * c->elem, cudaMemcpyDeviceToDevice,
                                c->stream) != cudaSuccess)
                return THIIM_ERR_CUDA;
        }
    }
    if (finalize_norms(c->partials, last_ctas, c->norms, c->stream) != cudaSuccess) return THIIM_ERR_CUDA;
    c->have_norm = true;
    return THIIM_OK;
}

int thiim_residual(thiim_ctx *c, double *rel_residual) {
    if (!c || !rel_residual) return THIIM_ERR_ARG;
    if (!c->have_norm) return THIIM_ERR_STATE;
    double h[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(h, c->norms, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return THIIM_ERR_CUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return THIIM_ERR_CUDA;
    if (!isfinite(h[0]) || !isfinite(h[1])) return THIIM_ERR_NONFINITE;
    *rel_residual = h[1] > 0.0 ? sqrt(h[0] / h[1]) : 0.0;
    return THIIM_OK;
}

int thiim_build_coeffs(thiim_ctx *c, const void *eps_r, const double *sigma_pml_e,
                       const double *sigma_pml_h, double omega, double tau, int k_s, double amp_re,
                       double amp_im, void *const coeff[THIIM_N_COEFFS]) {
    const double jones[4] = {amp_re, amp_im, 0.0, 0.0};
    return thiim_build_coeffs_jones(c, eps_r, sigma_pml_e, sigma_pml_h, omega, tau, k_s, jones, coeff);
}

int thiim_build_coeffs_jones(thiim_ctx *c, const void *eps_r, const double *sigma_pml_e,
                             const double *sigma_pml_h, double omega, double tau, int k_s,
                             const double jones[4], void *const coeff[THIIM_N_COEFFS]) {
    if (!c || !eps_r || !coeff || !jones) return THIIM_ERR_ARG;
    if (!aligned(eps_r, 16)) return THIIM_ERR_ALIGN;
    for (int i = 0; i < THIIM_N_COEFFS; ++i) {
        if (!coeff[i]) return THIIM_ERR_ARG;
        if (!aligned(coeff[i], c->elem)) return THIIM_ERR_ALIGN;
    }
    BuildArgs a;
    int st = prepare_build(c, sigma_pml_e, sigma_pml_h, omega, tau, k_s, jones, &a);
    if (st) return st;
    a.eps = (const double2 *)eps_r;
    memcpy(a.co, coeff, sizeof(a.co));
    const int threads = 256;
    long blocks = (long)((c->n_cells + threads - 1) / threads);
    if (blocks > 32L * c->num_sms) blocks = 32L * c->num_sms;
    c->pair_dirty = true;
    if (c->precision != THIIM_C64)
        build_coeffs_kernel<double2><<<(unsigned)blocks, threads, 0, c->stream>>>(a);
    else
        build_coeffs_kernel<float2><<<(unsigned)blocks, threads, 0, c->stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
    return read_build_flag(c);
}

int thiim_build_material_table(thiim_ctx *c, int n_mat, const double *eps_mat, const double *sigma_pml_e,
                               const double *sigma_pml_h, double omega, double tau, int k_s,
                               const double jones[4], void *table) {
    if (!c || !eps_mat || !table || !jones || n_mat < 1 || n_mat > THIIM_MAX_MATERIALS) return THIIM_ERR_ARG;
    if ((long long)n_mat * c->nz > 0x7FFFFFFFLL) return THIIM_ERR_ARG;   // table rows are indexed as int
    if (!aligned(table, c->elem)) return THIIM_ERR_ALIGN;
    for (int m = 0; m < 2 * n_mat; ++m)
        if (!isfinite(eps_mat[m])) return THIIM_ERR_ARG;
    for (int m = 0; m < n_mat; ++m)
        if (eps_mat[2 * m] == 0.0) return THIIM_ERR_ARG;
    BuildArgs a;
    int st = prepare_build(c, sigma_pml_e, sigma_pml_h, omega, tau, k_s, jones, &a);
    if (st) return st;
    if (!c->mat_eps && cudaMalloc(&c->mat_eps, 2 * THIIM_MAX_MATERIALS * sizeof(double)) != cudaSuccess)
        return THIIM_ERR_NOMEM;
    if (cudaMemcpyAsync(c->mat_eps, eps_mat, 2 * (size_t)n_mat * sizeof(double), cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return THIIM_ERR_CUDA;
    a.eps = (const double2 *)c->mat_eps;
    const int threads = 256;
    const int rows = n_mat * c->nz;
    const int blocks = (rows + threads - 1) / threads;
    c->pair_table_dirty = true;
    if (c->precision != THIIM_C64)
        build_table_kernel<double2><<<blocks, threads, 0, c->stream>>>(a, n_mat, table);
    else
        build_table_kernel<float2><<<blocks, threads, 0, c->stream>>>(a, n_mat, table);
    if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
    return read_build_flag(c);
}

void thiim_destroy(thiim_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < THIIM_N_FIELDS; ++i)
        if (c->alt[i]) cudaFree(c->alt[i]);
    for (int i = 0; i < THIIM_N_COEFFS; ++i)
        if (c->pair_co[i]) cudaFree(c->pair_co[i]);
    for (int i = 0; i < THIIM_N_FIELDS; ++i)
        if (c->mix_r[i]) cudaFree(c->mix_r[i]);
    for (int i = 0; i < 6; ++i) {
        if (c->adj_lh[i]) cudaFree(c->adj_lh[i]);
        if (c->adj_w[i]) cudaFree(c->adj_w[i]);
    }
    for (int m = 0; m < THIIM_MAX_ADJOINT_SEGMENT; ++m)
        for (int i = 0; i < THIIM_N_FIELDS; ++i)
            if (c->adj_states[m][i]) cudaFree(c->adj_states[m][i]);
    if (c->pair_table) cudaFree(c->pair_table);
    if (c->mat_eps) cudaFree(c->mat_eps);
    if (c->partials) cudaFree(c->partials);
    if (c->norms) cudaFree(c->norms);
    if (c->power) cudaFree(c->power);
    if (c->adj_norms) cudaFree(c->adj_norms);
    if (c->pml) cudaFree(c->pml);
    if (c->flag) cudaFree(c->flag);
    delete c;
}

}  // extern "C"
