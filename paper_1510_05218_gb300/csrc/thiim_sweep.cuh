// Fused THIIM E/H sweep (one iteration per launch), templated on precision.
//
// One iteration of the paper's scheme (Sec. I-A, Eqs. 3-7) is the six H split
// updates reading E^n followed by the six E split updates reading the new H
// (Listings 1-2 give two of the twelve).  This kernel streams along z (the
// outer dimension, as the wavefront of Sec. II-B does) and fuses both
// half-steps with a one-plane lag: at plane step k it forms H^{n+1/2}(k),
// which needs E^n at k and k-1, and then E^{n+1}(k-1), which needs the new H
// at k-1 and k.  Each CTA owns a TX x TY column of cells (x fastest) and a
// chunk of planes; it recomputes the new H on a one-cell halo at +x and +y
// (the E update reads H at +1) instead of exchanging it, and reads E^n on a
// one-cell halo at -x and -y.  Reads come from one field set and writes go to
// the other (ping-pong), so CTAs never wait on one another.
//
// Per cell and iteration the compulsory traffic is 40 arrays read (12 fields
// + 28 coefficients) and 12 written: 52 x 16 B = 832 B in FP64 and 416 B in
// FP32 (the paper's naive code moves 1344 B, Eq. 8).
//
// The arithmetic is a policy A (thiim_arith.cuh): native FP64, native FP32,
// or FP32 pairs on complex128 data.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "thiim_arith.cuh"

namespace thiim {

// Field order: Hxy Hxz Hyx Hyz Hzx Hzy Exy Exz Eyx Eyz Ezx Ezy.
enum { HXY, HXZ, HYX, HYZ, HZX, HZY, EXY, EXZ, EYX, EYZ, EZX, EZY };
// Coefficient order: t[12], c[12], SrcHxy, SrcHyx, SrcExy, SrcEyx.
enum { T0 = 0, C0 = 12, SRC_HXY = 24, SRC_HYX = 25, SRC_EXY = 26, SRC_EYX = 27 };

struct SweepArgs {
    const void *src[12];   // x^n
    void *dst[12];         // x^{n+1}
    const void *co[28];
    int nx, ny, nz;
    unsigned bc;           // bit 0/1/2: periodic x/y/z
    int zchunk;            // planes per CTA
    int tiles_x;           // CTAs along x
    double *partials;      // 2 doubles per CTA (|dF|^2, |F|^2) or nullptr
    const void *xsrc[12];  // SWEEP_CORRECT: per-split source arrays replacing Src
    // Material-table coefficients (the compressed variant): coefficient ci of
    // cell p on plane k is table[(mat[p] * nz + k) * 28 + ci].
    const unsigned char *mat;
    const void *table;
};

// Where the coefficients of one cell come from: element p of each of the 28
// arrays, or one 28-entry row of the (material, plane) table.
template <typename A, bool TBL>
struct CoefAt {
    size_t base;
    __device__ __forceinline__ CoefAt(const SweepArgs &a, size_t p, int k) {
        base = TBL ? ((size_t)a.mat[p] * a.nz + k) * 28 : p;
    }
    __device__ __forceinline__ typename A::Z get(const SweepArgs &a, int ci) const {
        return TBL ? A::ld_coef(a.table, base + ci) : A::ld_coef(a.co[ci], base);
    }
};

// Phase A loads E^n with L2 evict_last priority: the E update reads the
// same lines again one plane step later (and the neighbouring tiles read the
// halo rows), while most other lines are read once.  Measured at 512^3: pair
// +3-4 %, complex64 +0.6 %.  Marking the H phase's shared rows evict_last or
// once-used coefficient lines evict_first was slower.
#ifndef THIIM_L2_HINT_A
#define THIIM_L2_HINT_A 1
#endif

// Sweep modes.
//   SWEEP_PLAIN    dst <- one iteration of src.
//   SWEEP_DEFECT   dst <- (one iteration of src) - src, stored as complex64:
//                  the defect r = F(x) - x of the defect-correction restart.
//                  Where the two splits of a component have bit-identical t
//                  and c (everywhere outside the absorbing layers) their
//                  difference is an undamped mode that no full field sees;
//                  the pair's defect is stored balanced, (r_a + r_b)/2 each,
//                  which keeps the full-field defect r_a + r_b and keeps the
//                  complex64 correction from carrying that large, never
//                  decaying part (whose FP32 cancellation would otherwise
//                  set a floor under the FP64 residual).
//   SWEEP_CORRECT  dst <- M src + xsrc: the correction iteration
//                  delta <- M delta + r, where M is the linear part of one
//                  iteration (no Src).  r is added to what is stored only; the
//                  E update reads the new H *without* r_H, otherwise the H
//                  defect would leak into E through the curl a second time.
enum { SWEEP_PLAIN = 0, SWEEP_DEFECT = 1, SWEEP_CORRECT = 2 };

template <typename Z> struct Vec3 { Z x, y, z; };

// Map a halo coordinate g in [-1, n] into the grid; false if outside a
// non-periodic edge.
__device__ __forceinline__ bool wrap(int &g, int n, bool periodic) {
    if (g < 0) { if (!periodic) return false; g += n; }
    else if (g >= n) { if (!periodic) return false; g -= n; }
    return true;
}


template <typename A, int MODE, bool TBL = false>
struct SplitIO {
    typedef typename A::Z Z;
    // t x + c d (+ Src if the split has a source array; none in SWEEP_CORRECT).
    // The result feeds the full-field sums that the E update reads.
    __device__ static __forceinline__ Z update(const SweepArgs &a, int s, int src_coef, const CoefAt<A, TBL> &cr,
                                               Z x, Z d) {
        const Z t = cr.get(a, T0 + s), c = cr.get(a, C0 + s);
        if (MODE != SWEEP_CORRECT && src_coef >= 0) return A::upd_src(x, t, c, d, cr.get(a, src_coef));
        return A::upd(x, t, c, d);
    }
    // Store splits s and s+1 (the two parts of one component).
    __device__ static __forceinline__ void store_pair(const SweepArgs &a, int s, size_t p, Z va, Z olda, Z vb, Z oldb) {
        if (MODE == SWEEP_DEFECT) {
            double ar = A::re(va) - A::re(olda), ai = A::im(va) - A::im(olda);
            double br = A::re(vb) - A::re(oldb), bi = A::im(vb) - A::im(oldb);
            const Z ta = A::ld_coef(a.co[T0 + s], p), tb = A::ld_coef(a.co[T0 + s + 1], p);
            const Z ca = A::ld_coef(a.co[C0 + s], p), cb = A::ld_coef(a.co[C0 + s + 1], p);
            if (A::re(ta) == A::re(tb) && A::im(ta) == A::im(tb) && A::re(ca) == A::re(cb) && A::im(ca) == A::im(cb)) {
                ar = br = 0.5 * (ar + br);
                ai = bi = 0.5 * (ai + bi);
            }
            stg_as<float2>(a.dst[s], p, make_float2((float)ar, (float)ai));
            stg_as<float2>(a.dst[s + 1], p, make_float2((float)br, (float)bi));
        } else {
            store(a, s, p, va, olda);
            store(a, s + 1, p, vb, oldb);
        }
    }
    // Store the new value of split s (plus xsrc[s] in SWEEP_CORRECT; minus
    // the old value, as complex64, in SWEEP_DEFECT).
    __device__ static __forceinline__ void store(const SweepArgs &a, int s, size_t p, Z v, Z old) {
        if (MODE == SWEEP_CORRECT) {
            A::st_field(a.dst[s], p, A::add(v, A::ld_coef(a.xsrc[s], p)));
        } else if (MODE == SWEEP_DEFECT) {
            stg_as<float2>(a.dst[s], p, make_float2((float)(A::re(v) - A::re(old)), (float)(A::im(v) - A::im(old))));
        } else {
            A::st_field(a.dst[s], p, v);
        }
    }
};

// One CTA's share of an iteration: the TX x TY column `tile` over the z
// chunk `chunk`.  partial_out (2 doubles) receives the CTA's |dF|^2, |F|^2
// when non-null.  Used by the per-problem kernel below and by the batched
// persistent kernel (thiim_batch.cu).
template <typename A, int TX, int TY, int NT, int MODE, bool TBL = false>
__device__ __forceinline__ void sweep_tile(const SweepArgs &a, int tile, int chunk, double *partial_out) {
    typedef typename A::Z Z;
    typedef SplitIO<A, MODE, TBL> IO;
    constexpr int EW = TX + 2, EH = TY + 2;   // E^n region: -1 .. TX (x), -1 .. TY (y)
    constexpr int HW = TX + 1, HH = TY + 1;   // new-H region: 0 .. TX, 0 .. TY
    __shared__ Vec3<Z> sE[2][EH][EW];         // full E^n at planes k (cur) and k-1
    __shared__ Vec3<Z> sH[2][HH][HW];         // full new H at planes k (cur) and k-1
    __shared__ double red[2][NT / 32];

    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool px = a.bc & 1u, py = a.bc & 2u, pz = a.bc & 4u;
    const int i0 = (tile % a.tiles_x) * TX;
    const int j0 = (tile / a.tiles_x) * TY;
    const int nix = min(TX, nx - i0), niy = min(TY, ny - j0);
    const int z0 = chunk * a.zchunk;
    const int z1 = min(z0 + a.zchunk, nz);
    const size_t plane = (size_t)nx * ny;
    const int ew = nix + 2, ecount = (nix + 2) * (niy + 2);
    const int hw = nix + 1, hcount = (nix + 1) * (niy + 1);
    const int tcount = nix * niy;
    const bool want_norm = partial_out != nullptr;
    typename A::Acc acc_d = A::acc_zero(), acc_x = A::acc_zero();

    const uint64_t pol_keep = THIIM_L2_HINT_A ? l2_evict_last() : 0;
    auto ld_e_first = [&](int s, size_t p) {
        return THIIM_L2_HINT_A ? A::ld_field_hint(a.src[s], p, pol_keep) : A::ld_field(a.src[s], p);
    };

    // Phase A: full E^n on the E region of plane k into sE[b].
    auto load_E = [&](int k, int b) {
        bool zin = true;
        int kk = k;
        if (kk < 0 || kk >= nz) { if (pz) kk = (kk + nz) % nz; else zin = false; }
        for (int w = threadIdx.x; w < ecount; w += NT) {
            const int tx = w % ew, ty = w / ew;
            int gx = i0 - 1 + tx, gy = j0 - 1 + ty;
            Vec3<Z> f;
            f.x = f.y = f.z = A::zero();
            if (zin && wrap(gx, nx, px) && wrap(gy, ny, py)) {
                const size_t p = (size_t)kk * plane + (size_t)gy * nx + gx;
                f.x = A::add(ld_e_first(EXY, p), ld_e_first(EXZ, p));
                f.y = A::add(ld_e_first(EYX, p), ld_e_first(EYZ, p));
                f.z = A::add(ld_e_first(EZX, p), ld_e_first(EZY, p));
            }
            sE[b][ty][tx] = f;
        }
    };

    // L1 prefetch of what the next phase reads once from DRAM, issued before
    // the barrier that precedes that phase, so that its latency overlaps the
    // wait for the slowest warp (A::l1_prefetch >= 1: phase C's 14 E
    // coefficients; >= 2: also phase B's 14 H coefficients and 6 old H
    // splits).  No registers are held across the barrier.  Measured at
    // 512^3: FP32 pairs +3.4 % and FP64 +2.1 % at level 2; complex64 +0.4 %
    // at level 1 and 8 % slower at level 2 (its five CTAs per SM leave less
    // L1 per CTA).  Holding phase C's coefficients in registers instead
    // spilled and was 25 % slower (pairs).
    constexpr int PF = TBL ? 0 : A::l1_prefetch;
    auto prefetch_l1 = [](const void *base, size_t p) {
        asm volatile("prefetch.L1 [%0];" ::"l"((const char *)base + p * sizeof(Z)));
    };

    int cur = 0;
    load_E(z0 - 1, 1);            // E^n at plane z0-1 (zero below a Dirichlet edge)

    for (int k = z0; k <= z1; ++k) {
        const bool beyond = (k >= nz) && !pz;      // H above the top plane reads as zero
        const int kk = (k >= nz) ? k - nz : k;
        const int prev = cur ^ 1;
        if (!beyond) load_E(k, cur);
        if (PF >= 2 && !beyond) {
            for (int w = threadIdx.x; w < hcount; w += NT) {
                int gx = i0 + w % hw, gy = j0 + w / hw;
                if (!(wrap(gx, nx, px) && wrap(gy, ny, py))) continue;
                const size_t p = (size_t)kk * plane + (size_t)gy * nx + gx;
#pragma unroll
                for (int s = 0; s < 6; ++s) {
                    prefetch_l1(a.co[T0 + HXY + s], p);
                    prefetch_l1(a.co[C0 + HXY + s], p);
                    prefetch_l1(a.src[HXY + s], p);
                }
                if (MODE != SWEEP_CORRECT) {
                    prefetch_l1(a.co[SRC_HXY], p);
                    prefetch_l1(a.co[SRC_HYX], p);
                }
            }
        }
        __syncthreads();

        // Phase B: new H at plane k on the H region (tile plus +x/+y halo).
        for (int w = threadIdx.x; w < hcount; w += NT) {
            const int hx = w % hw, hy = w / hw;
            int gx = i0 + hx, gy = j0 + hy;
            Vec3<Z> hn;
            hn.x = hn.y = hn.z = A::zero();
            if (!beyond && wrap(gx, nx, px) && wrap(gy, ny, py)) {
                const size_t p = (size_t)kk * plane + (size_t)gy * nx + gx;
                const Vec3<Z> e0 = sE[cur][hy + 1][hx + 1];
                const Vec3<Z> exm = sE[cur][hy + 1][hx];
                const Vec3<Z> eym = sE[cur][hy][hx + 1];
                const Vec3<Z> ezm = sE[prev][hy + 1][hx + 1];
                // backward differences; the curl sign is folded into the order
                const Z dHxy = A::sub(e0.y, ezm.y);   // +dz Ey
                const Z dHxz = A::sub(eym.z, e0.z);   // -dy Ez
                const Z dHyx = A::sub(ezm.x, e0.x);   // -dz Ex
                const Z dHyz = A::sub(e0.z, exm.z);   // +dx Ez
                const Z dHzx = A::sub(e0.x, eym.x);   // +dy Ex
                const Z dHzy = A::sub(exm.y, e0.y);   // -dx Ey
                const Z oxy = A::ld_field(a.src[HXY], p), oxz = A::ld_field(a.src[HXZ], p);
                const Z oyx = A::ld_field(a.src[HYX], p), oyz = A::ld_field(a.src[HYZ], p);
                const Z ozx = A::ld_field(a.src[HZX], p), ozy = A::ld_field(a.src[HZY], p);
                const CoefAt<A, TBL> cr(a, p, kk);
                const Z nxy = IO::update(a, HXY, SRC_HXY, cr, oxy, dHxy);
                const Z nxz = IO::update(a, HXZ, -1, cr, oxz, dHxz);
                const Z nyx = IO::update(a, HYX, SRC_HYX, cr, oyx, dHyx);
                const Z nyz = IO::update(a, HYZ, -1, cr, oyz, dHyz);
                const Z nzx = IO::update(a, HZX, -1, cr, ozx, dHzx);
                const Z nzy = IO::update(a, HZY, -1, cr, ozy, dHzy);
                hn.x = A::add(nxy, nxz);
                hn.y = A::add(nyx, nyz);
                hn.z = A::add(nzx, nzy);
                if (hx < nix && hy < niy && k < z1) {
                    IO::store_pair(a, HXY, p, nxy, oxy, nxz, oxz);
                    IO::store_pair(a, HYX, p, nyx, oyx, nyz, oyz);
                    IO::store_pair(a, HZX, p, nzx, ozx, nzy, ozy);
                    if (want_norm) {
                        A::acc_d3(acc_d, hn.x, A::add(oxy, oxz), hn.y, A::add(oyx, oyz), hn.z, A::add(ozx, ozy));
                        A::acc_n3(acc_x, hn.x, hn.y, hn.z);
                    }
                }
            }
            sH[cur][hy][hx] = hn;
        }
        if (PF >= 1 && k > z0) {
            for (int w = threadIdx.x; w < tcount; w += NT) {
                const size_t p = (size_t)(k - 1) * plane + (size_t)(j0 + w / nix) * nx + (i0 + w % nix);
#pragma unroll
                for (int s = 0; s < 6; ++s) {
                    prefetch_l1(a.co[T0 + EXY + s], p);
                    prefetch_l1(a.co[C0 + EXY + s], p);
                }
                if (MODE != SWEEP_CORRECT) {
                    prefetch_l1(a.co[SRC_EXY], p);
                    prefetch_l1(a.co[SRC_EYX], p);
                }
            }
        }
        __syncthreads();

        // Phase C: new E at plane k-1 on the tile (needs new H at k-1 and k).
        if (k > z0) {
            const int ke = k - 1;
            for (int w = threadIdx.x; w < tcount; w += NT) {
                const int ex = w % nix, ey = w / nix;
                const int gx = i0 + ex, gy = j0 + ey;
                const size_t p = (size_t)ke * plane + (size_t)gy * nx + gx;
                const Vec3<Z> h0 = sH[prev][ey][ex];
                const Vec3<Z> hxp = sH[prev][ey][ex + 1];
                const Vec3<Z> hyp = sH[prev][ey + 1][ex];
                const Vec3<Z> hzp = sH[cur][ey][ex];
                // forward differences with the curl sign folded in
                const Z dExy = A::sub(h0.y, hzp.y);   // -dz Hy
                const Z dExz = A::sub(hyp.z, h0.z);   // +dy Hz
                const Z dEyx = A::sub(hzp.x, h0.x);   // +dz Hx
                const Z dEyz = A::sub(h0.z, hxp.z);   // -dx Hz
                const Z dEzx = A::sub(h0.x, hyp.x);   // -dy Hx
                const Z dEzy = A::sub(hxp.y, h0.y);   // +dx Hy
                const Z oxy = A::ld_field(a.src[EXY], p), oxz = A::ld_field(a.src[EXZ], p);
                const Z oyx = A::ld_field(a.src[EYX], p), oyz = A::ld_field(a.src[EYZ], p);
                const Z ozx = A::ld_field(a.src[EZX], p), ozy = A::ld_field(a.src[EZY], p);
                const CoefAt<A, TBL> cr(a, p, ke);
                const Z nxy = IO::update(a, EXY, SRC_EXY, cr, oxy, dExy);
                const Z nxz = IO::update(a, EXZ, -1, cr, oxz, dExz);
                const Z nyx = IO::update(a, EYX, SRC_EYX, cr, oyx, dEyx);
                const Z nyz = IO::update(a, EYZ, -1, cr, oyz, dEyz);
                const Z nzx = IO::update(a, EZX, -1, cr, ozx, dEzx);
                const Z nzy = IO::update(a, EZY, -1, cr, ozy, dEzy);
                IO::store_pair(a, EXY, p, nxy, oxy, nxz, oxz);
                IO::store_pair(a, EYX, p, nyx, oyx, nyz, oyz);
                IO::store_pair(a, EZX, p, nzx, ozx, nzy, ozy);
                if (want_norm) {
                    const Z fx = A::add(nxy, nxz), fy = A::add(nyx, nyz), fz = A::add(nzx, nzy);
                    A::acc_d3(acc_d, fx, A::add(oxy, oxz), fy, A::add(oyx, oyz), fz, A::add(ozx, ozy));
                    A::acc_n3(acc_x, fx, fy, fz);
                }
            }
        }
        cur = prev;
    }

    if (want_norm) {
        // CTA reduction in FP64 in a fixed order, then one partial pair per CTA.
        double sd = A::acc_value(acc_d), sx = A::acc_value(acc_x);
        for (int o = 16; o > 0; o >>= 1) {
            sd += __shfl_down_sync(0xffffffffu, sd, o);
            sx += __shfl_down_sync(0xffffffffu, sx, o);
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) { red[0][warp] = sd; red[1][warp] = sx; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double d = 0.0, x = 0.0;
            for (int i = 0; i < NT / 32; ++i) { d += red[0][i]; x += red[1][i]; }
            partial_out[0] = d;
            partial_out[1] = x;
        }
    }
}

template <typename A, int TX, int TY, int NT, int MINB, int MODE = SWEEP_PLAIN, bool TBL = false>
__global__ void __launch_bounds__(NT, (MINB > 0 ? MINB : (NT == 256 ? A::min_blocks : 1)))
sweep_kernel(const SweepArgs a) {
    const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    sweep_tile<A, TX, TY, NT, MODE, TBL>(a, blockIdx.x, blockIdx.y, a.partials ? a.partials + 2 * cta : nullptr);
}

}  // namespace thiim
