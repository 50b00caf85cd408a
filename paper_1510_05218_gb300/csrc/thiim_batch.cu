// Batched THIIM solves: many independent problems of uneven size advanced by
// one persistent launch per iteration (thiim_batch_iterate).
//
// A spectrum sweep (the paper's application needs 80-160 runs per cell,
// Sec. VI) is many small independent solves; launching each one separately
// leaves most SMs idle on the small grids.  Here every active solve's work is
// cut into items — one (tile column, z chunk) of one solve — and a grid of
// exactly as many CTAs as fit on the GPU walks the item list with a fixed
// stride, so CTAs move from one solve to the next without a launch.  Items
// read their solve's descriptor (field/coefficient pointers, sizes) into
// shared memory.  No CTA waits on another: each iteration is still one
// launch with the ping-pong field sets.
//
// Between convergence checks the `check_every` launches (plus the per-solve
// norm reduction) run as one captured CUDA graph.  The item list, its count
// and the descriptors live in device memory, so the same graph stays valid
// when converged solves drop out of the list.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "thiim_ctx.h"

using namespace thiim;

// z planes per batch item (every solve).
#ifndef THIIM_BATCH_ZCHUNK
#define THIIM_BATCH_ZCHUNK 32
#endif

namespace {

struct BatchDesc {
    void *f[2][THIIM_N_FIELDS];     // field sets: [0] the caller's, [1] the library's
    const void *co[THIIM_N_COEFFS];
    int nx, ny, nz;
    unsigned bc;
    int zchunk, tiles_x, tiles;
};

struct BatchList {
    const BatchDesc *desc;          // one per solve
    const int2 *items;              // (solve, local item) for the active solves
    const int *n_items;             // device scalar
    double *partials;               // 2 doubles per item
};

template <typename A, int MODE>
__global__ void __launch_bounds__(SWEEP_NT, Tile<A>::MINB)
batch_kernel(const BatchList L, int parity, int want_norm) {
    __shared__ SweepArgs sa;
    const int n = *L.n_items;
    for (int item = blockIdx.x; item < n; item += gridDim.x) {
        const int2 it = L.items[item];
        const BatchDesc &d = L.desc[it.x];
        if (threadIdx.x < THIIM_N_FIELDS) {
            sa.src[threadIdx.x] = d.f[parity][threadIdx.x];
            sa.dst[threadIdx.x] = d.f[parity ^ 1][threadIdx.x];
        }
        if (threadIdx.x < THIIM_N_COEFFS) sa.co[threadIdx.x] = d.co[threadIdx.x];
        if (threadIdx.x == 0) {
            sa.nx = d.nx; sa.ny = d.ny; sa.nz = d.nz;
            sa.bc = d.bc;
            sa.zchunk = d.zchunk;
            sa.tiles_x = d.tiles_x;
            sa.partials = nullptr;
        }
        __syncthreads();
        sweep_tile<A, Tile<A>::TX, Tile<A>::TY, SWEEP_NT, MODE>(sa, it.y % d.tiles, it.y / d.tiles,
                                                          want_norm ? L.partials + 2 * (size_t)item : nullptr);
        __syncthreads();   // sa and the tile's shared arrays are reused by the next item
    }
}

// Norms of solve b: sum of its items' partials (fixed order).
__global__ void batch_finalize(const int *first_item, const int *n_items_of, const double *partials, double *norms,
                               int nb) {
    const int b = blockIdx.x;
    if (b >= nb) return;
    __shared__ double sd[256], sx[256];
    double dsum = 0.0, xsum = 0.0;
    const int f = first_item[b], n = n_items_of[b];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        dsum += partials[2 * (size_t)(f + i)];
        xsum += partials[2 * (size_t)(f + i) + 1];
    }
    sd[threadIdx.x] = dsum;
    sx[threadIdx.x] = xsum;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) { sd[threadIdx.x] += sd[threadIdx.x + o]; sx[threadIdx.x] += sx[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0 && n > 0) { norms[2 * b] = sd[0]; norms[2 * b + 1] = sx[0]; }
}

struct ConvArgs {
    const float4 *src[THIIM_N_FIELDS];
    double2 *dst[THIIM_N_FIELDS];
};
// FP32 pairs -> complex128 (may run in place: each element is read, then written).
__global__ void pairs_to_c128(const ConvArgs a, size_t n) {
    const float4 *s = a.src[blockIdx.y];
    double2 *d = a.dst[blockIdx.y];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = s[i];
        d[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
}

cudaError_t launch_batch(int precision, bool first_pair, const BatchList &L, int grid, int parity, int want_norm,
                         cudaStream_t s) {
    if (precision == THIIM_C128)
        batch_kernel<Native<double>, SWEEP_PLAIN><<<grid, SWEEP_NT, 0, s>>>(L, parity, want_norm);
    else if (precision == THIIM_C64)
        batch_kernel<Native<float>, SWEEP_PLAIN><<<grid, SWEEP_NT, 0, s>>>(L, parity, want_norm);
    else if (first_pair)
        batch_kernel<PairArith<0, 1>, SWEEP_PLAIN><<<grid, SWEEP_NT, 0, s>>>(L, parity, want_norm);
    else
        batch_kernel<PairArith<1, 1>, SWEEP_PLAIN><<<grid, SWEEP_NT, 0, s>>>(L, parity, want_norm);
    return cudaGetLastError();
}

int resident_ctas(int precision, int num_sms) {
    int per_sm = 0;
    cudaError_t e;
    if (precision == THIIM_C128)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<Native<double>, SWEEP_PLAIN>, SWEEP_NT, 0);
    else if (precision == THIIM_C64)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<Native<float>, SWEEP_PLAIN>, SWEEP_NT, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<PairArith<1, 1>, SWEEP_PLAIN>, SWEEP_NT, 0);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * num_sms;
}

// Device buffers of one batch call, released on every exit path.
struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() { for (void *p : ptrs) cudaFree(p); }
    template <typename T> T *get(size_t count) {
        void *p = nullptr;
        if (cudaMalloc(&p, count * sizeof(T) + 16) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        ptrs.push_back(p);
        return (T *)p;
    }
};

// Split the coefficients of a THIIM_C128_PAIR context if they changed.
int ensure_pair_coeffs(thiim_ctx *c) {
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
    return THIIM_OK;
}

}  // namespace

extern "C" int thiim_batch_iterate(thiim_ctx *const ctx[], int nb, int max_iters, int check_every, double tol,
                                   int *iters_out, double *residual_out) {
    if (!ctx || nb < 1 || max_iters < 0 || check_every < 2 || (check_every & 1)) return THIIM_ERR_ARG;
    const int prec = ctx[0] ? ctx[0]->precision : -1;
    for (int b = 0; b < nb; ++b) {
        if (!ctx[b] || ctx[b]->precision != prec || ctx[b]->device != ctx[0]->device) return THIIM_ERR_ARG;
        if (!ctx[b]->have_fields || !ctx[b]->have_coeffs || ctx[b]->use_table) return THIIM_ERR_STATE;
    }
    cudaStream_t s = ctx[0]->stream;
    const bool pair = prec == THIIM_C128_PAIR;
    for (int b = 0; b < nb; ++b) {
        if (pair) {
            // splits run on each context's own stream; order them before the batch stream
            int st = ensure_pair_coeffs(ctx[b]);
            if (st) return st;
            if (ctx[b]->stream != s && cudaStreamSynchronize(ctx[b]->stream) != cudaSuccess) return THIIM_ERR_CUDA;
        }
        if (iters_out) iters_out[b] = 0;
        if (residual_out) residual_out[b] = -1.0;
    }
    if (max_iters == 0) return THIIM_OK;

    // Descriptors and the full item list (solve-major).
    std::vector<BatchDesc> desc(nb);
    std::vector<int> first(nb), count(nb);
    int total_items = 0;
    for (int b = 0; b < nb; ++b) {
        thiim_ctx *c = ctx[b];
        BatchDesc &d = desc[b];
        memset(&d, 0, sizeof(d));
        memcpy(d.f[0], c->user, sizeof(d.f[0]));
        memcpy(d.f[1], c->alt, sizeof(d.f[1]));
        memcpy(d.co, pair ? c->pair_co : c->coeff, sizeof(d.co));
        d.nx = c->nx; d.ny = c->ny; d.nz = c->nz;
        d.bc = c->bc;
        // the batch kernel's tile (compile time: Tile<A>; FP64 always on the tall tile)
        const int bty = c->precision == THIIM_C128 ? Tile<Native<double>>::TY : tile_h(c);
        d.tiles_x = tiles_x(c);
        d.tiles = d.tiles_x * ((c->ny + bty - 1) / bty);
        d.zchunk = c->nz < THIIM_BATCH_ZCHUNK ? c->nz : THIIM_BATCH_ZCHUNK;   // similar item sizes across solves
        const int chunks = (c->nz + d.zchunk - 1) / d.zchunk;
        first[b] = total_items;
        count[b] = d.tiles * chunks;
        total_items += count[b];
    }
    Scratch sc;
    BatchDesc *d_desc = sc.get<BatchDesc>(nb);
    int2 *d_items = sc.get<int2>(total_items);
    int *d_n = sc.get<int>(1);
    double *d_part = sc.get<double>(2 * (size_t)total_items);
    int *d_first = sc.get<int>(nb);
    int *d_count = sc.get<int>(nb);
    double *d_norms = sc.get<double>(2 * (size_t)nb);
    if (!d_desc || !d_items || !d_n || !d_part || !d_first || !d_count || !d_norms) return THIIM_ERR_NOMEM;
    if (cudaMemcpyAsync(d_desc, desc.data(), nb * sizeof(BatchDesc), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return THIIM_ERR_CUDA;

    std::vector<int> active(nb, 1), done(nb, 0);
    std::vector<int2> items;
    std::vector<int> h_first(nb), h_count(nb);
    // Rebuild the device item list for the active solves (synchronous: the
    // host vectors are reused right after).
    auto upload = [&]() -> int {
        items.clear();
        for (int b = 0; b < nb; ++b) {
            h_first[b] = (int)items.size();
            h_count[b] = active[b] ? count[b] : 0;
            if (!active[b]) continue;
            for (int i = 0; i < count[b]; ++i) items.push_back(make_int2(b, i));
        }
        const int n = (int)items.size();
        if ((n && cudaMemcpyAsync(d_items, items.data(), n * sizeof(int2), cudaMemcpyHostToDevice, s) != cudaSuccess) ||
            cudaMemcpyAsync(d_n, &n, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_first, h_first.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_count, h_count.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return THIIM_ERR_CUDA;
        return THIIM_OK;
    };
    int st = upload();
    if (st) return st;

    BatchList L;
    L.desc = d_desc;
    L.items = d_items;
    L.n_items = d_n;
    L.partials = d_part;
    const int grid = resident_ctas(prec, ctx[0]->num_sms);

    int iters = 0;
    int cur = 0;                       // field set holding the active solves' iterate
    std::vector<int> where(nb, 0);     // field set holding each solve's iterate
    std::vector<double> h_norms(2 * (size_t)nb);
    // Read the per-solve norms of the last iteration and retire solves that
    // reached tol (or max_iters).
    auto check = [&]() -> int {
        batch_finalize<<<nb, 256, 0, s>>>(d_first, d_count, d_part, d_norms, nb);
        if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
        return THIIM_OK;
    };
    auto retire = [&]() -> int {
        if (cudaMemcpyAsync(h_norms.data(), d_norms, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return THIIM_ERR_CUDA;
        bool changed = false;
        for (int b = 0; b < nb; ++b) {
            if (!active[b]) continue;
            done[b] = iters;
            where[b] = cur;
            const double dn = h_norms[2 * b], xn = h_norms[2 * b + 1];
            const double r = (isfinite(dn) && isfinite(xn)) ? (xn > 0.0 ? sqrt(dn / xn) : 0.0) : NAN;
            if (residual_out) residual_out[b] = r;
            if (!(r == r) || r <= tol || iters >= max_iters) { active[b] = 0; changed = true; }
        }
        return changed ? upload() : THIIM_OK;
    };
    if (pair) {    // first iteration: complex128 in, pairs out
        if (launch_batch(prec, true, L, grid, 0, max_iters == 1, s) != cudaSuccess) return THIIM_ERR_CUDA;
        cur = 1;
        iters = 1;
        if (max_iters == 1 && ((st = check()) || (st = retire()))) return st;
    }

    // One chunk of `check_every` iterations as a CUDA graph (starting in set `cur`).
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    struct GraphGuard {
        cudaGraphExec_t *e; cudaStream_t *c;
        ~GraphGuard() { if (*e) cudaGraphExecDestroy(*e); if (*c) cudaStreamDestroy(*c); }
    } guard{&exec, &cap};
    auto build_graph = [&]() -> int {
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return THIIM_ERR_CUDA;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return THIIM_ERR_CUDA;
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < check_every && e == cudaSuccess; ++i)
            e = launch_batch(prec, false, L, grid, cur ^ (i & 1), i == check_every - 1, cap);
        if (e == cudaSuccess) {
            batch_finalize<<<nb, 256, 0, cap>>>(d_first, d_count, d_part, d_norms, nb);
            e = cudaGetLastError();
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e != cudaSuccess || e2 != cudaSuccess || !g) { if (g) cudaGraphDestroy(g); return THIIM_ERR_CUDA; }
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        return e == cudaSuccess ? THIIM_OK : THIIM_ERR_CUDA;
    };

    while (iters < max_iters) {
        int n_active = 0;
        for (int b = 0; b < nb; ++b) n_active += active[b];
        if (!n_active) break;
        const int left = max_iters - iters;
        if (left >= check_every) {     // even length: `cur` is unchanged afterwards
            if (!exec && (st = build_graph())) return st;
            if (cudaGraphLaunch(exec, s) != cudaSuccess) return THIIM_ERR_CUDA;
            iters += check_every;
        } else {                       // a shorter last chunk: plain launches
            for (int i = 0; i < left; ++i)
                if (launch_batch(prec, false, L, grid, cur ^ (i & 1), i == left - 1, s) != cudaSuccess)
                    return THIIM_ERR_CUDA;
            if ((st = check())) return st;
            if (left & 1) cur ^= 1;
            iters += left;
        }
        if ((st = retire())) return st;
    }
    // Bring every solve's iterate into the caller's arrays as complex128/complex64.
    for (int b = 0; b < nb; ++b) {
        thiim_ctx *c = ctx[b];
        if (iters_out) iters_out[b] = done[b];
        if (pair) {
            ConvArgs a;
            for (int i = 0; i < THIIM_N_FIELDS; ++i) {
                a.src[i] = (const float4 *)desc[b].f[where[b]][i];
                a.dst[i] = (double2 *)c->user[i];
            }
            size_t blocks = (c->n_cells + 255) / 256;
            if (blocks > 2048) blocks = 2048;
            pairs_to_c128<<<dim3((unsigned)blocks, THIIM_N_FIELDS), 256, 0, s>>>(a, c->n_cells);
            if (cudaGetLastError() != cudaSuccess) return THIIM_ERR_CUDA;
        } else if (where[b] == 1) {
            for (int i = 0; i < THIIM_N_FIELDS; ++i)
                if (cudaMemcpyAsync(c->user[i], c->alt[i], c->n_cells * c->elem, cudaMemcpyDeviceToDevice, s) !=
                    cudaSuccess)
                    return THIIM_ERR_CUDA;
        }
        // the per-solve norms become the context's residual
        if (!c->norms && cudaMalloc(&c->norms, 2 * sizeof(double)) != cudaSuccess) return THIIM_ERR_NOMEM;
        if (cudaMemcpyAsync(c->norms, d_norms + 2 * b, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return THIIM_ERR_CUDA;
        c->have_norm = done[b] > 0;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return THIIM_ERR_CUDA;
    for (int b = 0; b < nb; ++b)
        if (residual_out && !(residual_out[b] == residual_out[b])) return THIIM_ERR_NONFINITE;
    return THIIM_OK;
}
