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
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace thiim {

template <typename R> struct cplx_of;
template <> struct cplx_of<double> { typedef double2 type; };
template <> struct cplx_of<float> { typedef float2 type; };

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
};

template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

// t*x + src + c*d  (d already carries the curl sign)
template <typename V>
__device__ __forceinline__ V upd_src(V x, V t, V c, V d, V s) {
    V r;
    r.x = fma(t.x, x.x, s.x); r.x = fma(-t.y, x.y, r.x); r.x = fma(c.x, d.x, r.x); r.x = fma(-c.y, d.y, r.x);
    r.y = fma(t.x, x.y, s.y); r.y = fma(t.y, x.x, r.y); r.y = fma(c.x, d.y, r.y); r.y = fma(c.y, d.x, r.y);
    return r;
}
template <typename V>
__device__ __forceinline__ V upd(V x, V t, V c, V d) {
    V r;
    r.x = t.x * x.x; r.x = fma(-t.y, x.y, r.x); r.x = fma(c.x, d.x, r.x); r.x = fma(-c.y, d.y, r.x);
    r.y = t.x * x.y; r.y = fma(t.y, x.x, r.y); r.y = fma(c.x, d.y, r.y); r.y = fma(c.y, d.x, r.y);
    return r;
}

template <typename V>
__device__ __forceinline__ V ldg(const void *base, size_t i) {
    return __ldg(reinterpret_cast<const V *>(base) + i);
}
template <typename V>
__device__ __forceinline__ void stg(void *base, size_t i, V v) {
    reinterpret_cast<V *>(base)[i] = v;
}

template <typename V> struct Vec3 { V x, y, z; };

// Map a halo coordinate g in [-1, n] into the grid; false if outside a
// non-periodic edge.
__device__ __forceinline__ bool wrap(int &g, int n, bool periodic) {
    if (g < 0) { if (!periodic) return false; g += n; }
    else if (g >= n) { if (!periodic) return false; g -= n; }
    return true;
}

template <typename R, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
sweep_kernel(const SweepArgs a) {
    typedef typename cplx_of<R>::type V;
    constexpr int EW = TX + 2, EH = TY + 2;   // E^n region: -1 .. TX (x), -1 .. TY (y)
    constexpr int HW = TX + 1, HH = TY + 1;   // new-H region: 0 .. TX, 0 .. TY
    __shared__ Vec3<V> sE[2][EH][EW];         // full E^n at planes k (cur) and k-1
    __shared__ Vec3<V> sH[2][HH][HW];         // full new H at planes k (cur) and k-1
    __shared__ double red[2][NT / 32];

    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool px = a.bc & 1u, py = a.bc & 2u, pz = a.bc & 4u;
    const int tile = blockIdx.x;
    const int i0 = (tile % a.tiles_x) * TX;
    const int j0 = (tile / a.tiles_x) * TY;
    const int nix = min(TX, nx - i0), niy = min(TY, ny - j0);
    const int z0 = blockIdx.y * a.zchunk;
    const int z1 = min(z0 + a.zchunk, nz);
    const size_t plane = (size_t)nx * ny;
    const int ew = nix + 2, ecount = (nix + 2) * (niy + 2);
    const int hw = nix + 1, hcount = (nix + 1) * (niy + 1);
    const int tcount = nix * niy;
    const bool want_norm = a.partials != nullptr;
    double acc_d = 0.0, acc_x = 0.0;

    // Phase A: full E^n on the E region of plane k into sE[b].
    auto load_E = [&](int k, int b) {
        bool zin = true;
        int kk = k;
        if (kk < 0 || kk >= nz) { if (pz) kk = (kk + nz) % nz; else zin = false; }
        for (int w = threadIdx.x; w < ecount; w += NT) {
            const int tx = w % ew, ty = w / ew;
            int gx = i0 - 1 + tx, gy = j0 - 1 + ty;
            Vec3<V> f;
            f.x.x = f.x.y = f.y.x = f.y.y = f.z.x = f.z.y = R(0);
            if (zin && wrap(gx, nx, px) && wrap(gy, ny, py)) {
                const size_t p = (size_t)kk * plane + (size_t)gy * nx + gx;
                f.x = cadd(ldg<V>(a.src[EXY], p), ldg<V>(a.src[EXZ], p));
                f.y = cadd(ldg<V>(a.src[EYX], p), ldg<V>(a.src[EYZ], p));
                f.z = cadd(ldg<V>(a.src[EZX], p), ldg<V>(a.src[EZY], p));
            }
            sE[b][ty][tx] = f;
        }
    };

    int cur = 0;
    load_E(z0 - 1, 1);            // E^n at plane z0-1 (zero below a Dirichlet edge)

    for (int k = z0; k <= z1; ++k) {
        const bool beyond = (k >= nz) && !pz;      // H above the top plane reads as zero
        const int kk = (k >= nz) ? k - nz : k;
        const int prev = cur ^ 1;
        if (!beyond) load_E(k, cur);
        __syncthreads();

        // Phase B: new H at plane k on the H region (tile plus +x/+y halo).
        for (int w = threadIdx.x; w < hcount; w += NT) {
            const int hx = w % hw, hy = w / hw;
            int gx = i0 + hx, gy = j0 + hy;
            Vec3<V> hn;
            hn.x.x = hn.x.y = hn.y.x = hn.y.y = hn.z.x = hn.z.y = R(0);
            if (!beyond && wrap(gx, nx, px) && wrap(gy, ny, py)) {
                const size_t p = (size_t)kk * plane + (size_t)gy * nx + gx;
                const Vec3<V> e0 = sE[cur][hy + 1][hx + 1];
                const Vec3<V> exm = sE[cur][hy + 1][hx];
                const Vec3<V> eym = sE[cur][hy][hx + 1];
                const Vec3<V> ezm = sE[prev][hy + 1][hx + 1];
                // backward differences; the curl sign is folded into the order
                const V dHxy = csub(e0.y, ezm.y);   // +dz Ey
                const V dHxz = csub(eym.z, e0.z);   // -dy Ez
                const V dHyx = csub(ezm.x, e0.x);   // -dz Ex
                const V dHyz = csub(e0.z, exm.z);   // +dx Ez
                const V dHzx = csub(e0.x, eym.x);   // +dy Ex
                const V dHzy = csub(exm.y, e0.y);   // -dx Ey
                const V oxy = ldg<V>(a.src[HXY], p), oxz = ldg<V>(a.src[HXZ], p);
                const V oyx = ldg<V>(a.src[HYX], p), oyz = ldg<V>(a.src[HYZ], p);
                const V ozx = ldg<V>(a.src[HZX], p), ozy = ldg<V>(a.src[HZY], p);
                const V nxy = upd_src(oxy, ldg<V>(a.co[T0 + HXY], p), ldg<V>(a.co[C0 + HXY], p), dHxy, ldg<V>(a.co[SRC_HXY], p));
                const V nxz = upd(oxz, ldg<V>(a.co[T0 + HXZ], p), ldg<V>(a.co[C0 + HXZ], p), dHxz);
                const V nyx = upd_src(oyx, ldg<V>(a.co[T0 + HYX], p), ldg<V>(a.co[C0 + HYX], p), dHyx, ldg<V>(a.co[SRC_HYX], p));
                const V nyz = upd(oyz, ldg<V>(a.co[T0 + HYZ], p), ldg<V>(a.co[C0 + HYZ], p), dHyz);
                const V nzx = upd(ozx, ldg<V>(a.co[T0 + HZX], p), ldg<V>(a.co[C0 + HZX], p), dHzx);
                const V nzy = upd(ozy, ldg<V>(a.co[T0 + HZY], p), ldg<V>(a.co[C0 + HZY], p), dHzy);
                hn.x = cadd(nxy, nxz);
                hn.y = cadd(nyx, nyz);
                hn.z = cadd(nzx, nzy);
                if (hx < nix && hy < niy && k < z1) {
                    stg(a.dst[HXY], p, nxy); stg(a.dst[HXZ], p, nxz);
                    stg(a.dst[HYX], p, nyx); stg(a.dst[HYZ], p, nyz);
                    stg(a.dst[HZX], p, nzx); stg(a.dst[HZY], p, nzy);
                    if (want_norm) {
                        const V dx = csub(hn.x, cadd(oxy, oxz));
                        const V dy = csub(hn.y, cadd(oyx, oyz));
                        const V dz = csub(hn.z, cadd(ozx, ozy));
                        acc_d += (double)dx.x * dx.x + (double)dx.y * dx.y + (double)dy.x * dy.x +
                                 (double)dy.y * dy.y + (double)dz.x * dz.x + (double)dz.y * dz.y;
                        acc_x += (double)hn.x.x * hn.x.x + (double)hn.x.y * hn.x.y + (double)hn.y.x * hn.y.x +
                                 (double)hn.y.y * hn.y.y + (double)hn.z.x * hn.z.x + (double)hn.z.y * hn.z.y;
                    }
                }
            }
            sH[cur][hy][hx] = hn;
        }
        __syncthreads();

        // Phase C: new E at plane k-1 on the tile (needs new H at k-1 and k).
        if (k > z0) {
            const int ke = k - 1;
            for (int w = threadIdx.x; w < tcount; w += NT) {
                const int ex = w % nix, ey = w / nix;
                const int gx = i0 + ex, gy = j0 + ey;
                const size_t p = (size_t)ke * plane + (size_t)gy * nx + gx;
                const Vec3<V> h0 = sH[prev][ey][ex];
                const Vec3<V> hxp = sH[prev][ey][ex + 1];
                const Vec3<V> hyp = sH[prev][ey + 1][ex];
                const Vec3<V> hzp = sH[cur][ey][ex];
                // forward differences with the curl sign folded in
                const V dExy = csub(h0.y, hzp.y);   // -dz Hy
                const V dExz = csub(hyp.z, h0.z);   // +dy Hz
                const V dEyx = csub(hzp.x, h0.x);   // +dz Hx
                const V dEyz = csub(h0.z, hxp.z);   // -dx Hz
                const V dEzx = csub(h0.x, hyp.x);   // -dy Hx
                const V dEzy = csub(hxp.y, h0.y);   // +dx Hy
                const V oxy = ldg<V>(a.src[EXY], p), oxz = ldg<V>(a.src[EXZ], p);
                const V oyx = ldg<V>(a.src[EYX], p), oyz = ldg<V>(a.src[EYZ], p);
                const V ozx = ldg<V>(a.src[EZX], p), ozy = ldg<V>(a.src[EZY], p);
                const V nxy = upd_src(oxy, ldg<V>(a.co[T0 + EXY], p), ldg<V>(a.co[C0 + EXY], p), dExy, ldg<V>(a.co[SRC_EXY], p));
                const V nxz = upd(oxz, ldg<V>(a.co[T0 + EXZ], p), ldg<V>(a.co[C0 + EXZ], p), dExz);
                const V nyx = upd_src(oyx, ldg<V>(a.co[T0 + EYX], p), ldg<V>(a.co[C0 + EYX], p), dEyx, ldg<V>(a.co[SRC_EYX], p));
                const V nyz = upd(oyz, ldg<V>(a.co[T0 + EYZ], p), ldg<V>(a.co[C0 + EYZ], p), dEyz);
                const V nzx = upd(ozx, ldg<V>(a.co[T0 + EZX], p), ldg<V>(a.co[C0 + EZX], p), dEzx);
                const V nzy = upd(ozy, ldg<V>(a.co[T0 + EZY], p), ldg<V>(a.co[C0 + EZY], p), dEzy);
                stg(a.dst[EXY], p, nxy); stg(a.dst[EXZ], p, nxz);
                stg(a.dst[EYX], p, nyx); stg(a.dst[EYZ], p, nyz);
                stg(a.dst[EZX], p, nzx); stg(a.dst[EZY], p, nzy);
                if (want_norm) {
                    const V fx = cadd(nxy, nxz), fy = cadd(nyx, nyz), fz = cadd(nzx, nzy);
                    const V dx = csub(fx, cadd(oxy, oxz));
                    const V dy = csub(fy, cadd(oyx, oyz));
                    const V dz = csub(fz, cadd(ozx, ozy));
                    acc_d += (double)dx.x * dx.x + (double)dx.y * dx.y + (double)dy.x * dy.x +
                             (double)dy.y * dy.y + (double)dz.x * dz.x + (double)dz.y * dz.y;
                    acc_x += (double)fx.x * fx.x + (double)fx.y * fx.y + (double)fy.x * fy.x +
                             (double)fy.y * fy.y + (double)fz.x * fz.x + (double)fz.y * fz.y;
                }
            }
        }
        cur = prev;
    }

    if (want_norm) {
        // CTA reduction in a fixed order, then one partial pair per CTA.
        for (int o = 16; o > 0; o >>= 1) {
            acc_d += __shfl_down_sync(0xffffffffu, acc_d, o);
            acc_x += __shfl_down_sync(0xffffffffu, acc_x, o);
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) { red[0][warp] = acc_d; red[1][warp] = acc_x; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double d = 0.0, x = 0.0;
            for (int i = 0; i < NT / 32; ++i) { d += red[0][i]; x += red[1][i]; }
            const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
            a.partials[2 * cta] = d;
            a.partials[2 * cta + 1] = x;
        }
    }
}

}  // namespace thiim
