// Temporal blocking: two THIIM iterations per pass over HBM.
//
// The paper decouples the sweep from memory bandwidth by updating a tile
// several times while it is in cache (diamond tiles along y with a wavefront
// along z, Sec. II, Figs. 2-4).  Here one CTA does the GPU analogue for two
// iterations: it streams its column along z and runs two staged iterations
// with a one-plane lag between them.  Stage 1 computes x^1 = F(x^0) on a
// region grown by the halo the second iteration needs — the new H on the
// tile + 1 cell (-x,-y) + 2 cells (+x,+y)... precisely:
//     E^0 full sums   on u in [-2, nix+1], v in [-2, niy+1]   (loaded)
//     H^1             on u in [-1, nix+1], v in [-1, niy+1]
//     E^1             on u in [-1, nix  ], v in [-1, niy  ]
//     H^2             on u in [ 0, nix  ], v in [ 0, niy  ]
//     E^2             on u in [ 0, nix-1], v in [ 0, niy-1]   (the tile; stored)
// (u, v relative to the tile origin).  x^1 never leaves shared memory; only
// x^2 is written.  At plane step k, stage 1 produces H^1(k) and E^1(k-1) and
// stage 2 produces H^2(k-1) and E^2(k-2).  Values outside a non-periodic
// edge are zero for every iterate, as in the single-iteration sweep.  Each
// cell's arithmetic is exactly that of two single sweeps, so the result is
// bit-identical to them.
//
// Per pass the CTA reads x^0 and the coefficients once (the second
// iteration's coefficients are re-read one or two plane steps later, from
// L2) and writes x^2 once: DRAM bytes per iteration roughly halve, at the
// price of ~16 % redundant arithmetic on the halo and 2 barriers per plane.
#pragma once

#include "thiim_sweep.cuh"

namespace thiim {

template <typename A, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT, 1)
sweep2_kernel(const SweepArgs a) {
    typedef typename A::Z Z;
    // region sizes (maximal tile)
    constexpr int W0 = TX + 4, H0 = TY + 4;   // E^0 sums      u,v in [-2, n+1]
    constexpr int W1 = TX + 3, H1 = TY + 3;   // H^1           u,v in [-1, n+1]
    constexpr int We = TX + 2, He = TY + 2;   // E^1           u,v in [-1, n]
    constexpr int W2 = TX + 1, H2 = TY + 1;   // H^2           u,v in [ 0, n]
    __shared__ Vec3<Z> sE0[2][H0][W0];        // full E^0, planes k, k-1
    __shared__ Vec3<Z> sH1[2][H1][W1];        // full H^1, planes k, k-1
    __shared__ Z sH1s[2][6][H2][W2];          // H^1 splits on the H^2 region, planes k, k-1
    __shared__ Vec3<Z> sE1[2][He][We];        // full E^1, planes k-1, k-2
    __shared__ Z sE1s[2][6][TY][TX];          // E^1 splits on the tile, planes k-1, k-2
    __shared__ Vec3<Z> sH2[2][H2][W2];        // full H^2, planes k-1, k-2
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
    const bool want_norm = a.partials != nullptr;
    typename A::Acc acc_d = A::acc_zero(), acc_x = A::acc_zero();

    // plane index inside the grid, or -1 outside a Dirichlet edge
    auto zin = [&](int k) -> int {
        if (k >= 0 && k < nz) return k;
        if (!pz) return -1;
        return ((k % nz) + nz) % nz;
    };
    // global cell of local (u, v) on plane kk, or -1 outside a Dirichlet edge
    auto cell = [&](int u, int v, int kk) -> long long {
        int gx = i0 + u, gy = j0 + v;
        if (kk < 0) return -1;
        if (gx < 0 || gx >= nx) { if (!px) return -1; gx = ((gx % nx) + nx) % nx; }
        if (gy < 0 || gy >= ny) { if (!py) return -1; gy = ((gy % ny) + ny) % ny; }
        return (long long)kk * plane + (long long)gy * nx + gx;
    };

    const int w0 = nix + 4, c0 = (nix + 4) * (niy + 4);
    const int w1 = nix + 3, c1 = (nix + 3) * (niy + 3);
    const int we = nix + 2, ce = (nix + 2) * (niy + 2);
    const int w2 = nix + 1, c2 = (nix + 1) * (niy + 1);
    const int ct = nix * niy;

    // Stage-0 load: full E^0 sums on the E^0 region of plane k into sE0[b].
    auto load_E0 = [&](int k, int b) {
        const int kk = zin(k);
        for (int w = threadIdx.x; w < c0; w += NT) {
            const int u = w % w0 - 2, v = w / w0 - 2;
            Vec3<Z> f;
            f.x = f.y = f.z = A::zero();
            const long long p = cell(u, v, kk);
            if (p >= 0) {
                f.x = A::add(A::ld_field(a.src[EXY], p), A::ld_field(a.src[EXZ], p));
                f.y = A::add(A::ld_field(a.src[EYX], p), A::ld_field(a.src[EYZ], p));
                f.z = A::add(A::ld_field(a.src[EZX], p), A::ld_field(a.src[EZY], p));
            }
            sE0[b][v + 2][u + 2] = f;
        }
    };

    // The H update of one cell from full-E sums at (own, -x, -y, -z) and the
    // old splits: the six new splits and their sums.
    struct HOut { Z s[6]; Vec3<Z> f; };
    auto h_update = [&](long long p, const Vec3<Z> &e0, const Vec3<Z> &exm, const Vec3<Z> &eym,
                        const Vec3<Z> &ezm, const Z o[6]) -> HOut {
        HOut r;
        r.s[0] = A::upd_src(o[0], A::ld_coef(a.co[T0 + HXY], p), A::ld_coef(a.co[C0 + HXY], p), A::sub(e0.y, ezm.y), A::ld_coef(a.co[SRC_HXY], p));
        r.s[1] = A::upd(o[1], A::ld_coef(a.co[T0 + HXZ], p), A::ld_coef(a.co[C0 + HXZ], p), A::sub(eym.z, e0.z));
        r.s[2] = A::upd_src(o[2], A::ld_coef(a.co[T0 + HYX], p), A::ld_coef(a.co[C0 + HYX], p), A::sub(ezm.x, e0.x), A::ld_coef(a.co[SRC_HYX], p));
        r.s[3] = A::upd(o[3], A::ld_coef(a.co[T0 + HYZ], p), A::ld_coef(a.co[C0 + HYZ], p), A::sub(e0.z, exm.z));
        r.s[4] = A::upd(o[4], A::ld_coef(a.co[T0 + HZX], p), A::ld_coef(a.co[C0 + HZX], p), A::sub(e0.x, eym.x));
        r.s[5] = A::upd(o[5], A::ld_coef(a.co[T0 + HZY], p), A::ld_coef(a.co[C0 + HZY], p), A::sub(exm.y, e0.y));
        r.f.x = A::add(r.s[0], r.s[1]);
        r.f.y = A::add(r.s[2], r.s[3]);
        r.f.z = A::add(r.s[4], r.s[5]);
        return r;
    };
    // The E update from full-H sums at (own, +x, +y, +z) and the old splits.
    auto e_update = [&](long long p, const Vec3<Z> &h0, const Vec3<Z> &hxp, const Vec3<Z> &hyp,
                        const Vec3<Z> &hzp, const Z o[6], Z out[6]) {
        out[0] = A::upd_src(o[0], A::ld_coef(a.co[T0 + EXY], p), A::ld_coef(a.co[C0 + EXY], p), A::sub(h0.y, hzp.y), A::ld_coef(a.co[SRC_EXY], p));
        out[1] = A::upd(o[1], A::ld_coef(a.co[T0 + EXZ], p), A::ld_coef(a.co[C0 + EXZ], p), A::sub(hyp.z, h0.z));
        out[2] = A::upd_src(o[2], A::ld_coef(a.co[T0 + EYX], p), A::ld_coef(a.co[C0 + EYX], p), A::sub(hzp.x, h0.x), A::ld_coef(a.co[SRC_EYX], p));
        out[3] = A::upd(o[3], A::ld_coef(a.co[T0 + EYZ], p), A::ld_coef(a.co[C0 + EYZ], p), A::sub(h0.z, hxp.z));
        out[4] = A::upd(o[4], A::ld_coef(a.co[T0 + EZX], p), A::ld_coef(a.co[C0 + EZX], p), A::sub(h0.x, hyp.x));
        out[5] = A::upd(o[5], A::ld_coef(a.co[T0 + EZY], p), A::ld_coef(a.co[C0 + EZY], p), A::sub(hxp.y, h0.y));
    };

    // prologue: E^0 at plane z0-2 (for H^1(z0-1)'s z difference)
    int b0 = 0;                       // sE0[b0] receives plane k
    load_E0(z0 - 2, 1);
    int bh = 0, be = 0;               // sH1/sH1s[bh] receive plane k; sE1/sE1s[be] receive plane k-1
    int b2 = 0;                       // sH2[b2] receives plane k-1

    // Per plane step two barriers: after A (E^0(k) loaded) and after BC
    // (H^1(k), E^1(k-1) complete).  B and C share a pass, as do D and E: the
    // E update of a cell needs the new H of the plane above at the same cell
    // only, which the same thread has just formed; its other inputs were
    // written before the last barrier.  The next step's A writes the E^0
    // buffer of plane k-1, which only B of this step read.
    for (int k = z0 - 1; k <= z1 + 1; ++k) {
        const int kk = zin(k);
        const int km = zin(k - 1);
        // ---- A: E^0(k) sums
        load_E0(k, b0);
        __syncthreads();
        // ---- BC: H^1(k) on the H^1 region (splits kept on the H^2 region);
        //      E^1(k-1) on the E^1 region (splits kept on the tile)
        for (int w = threadIdx.x; w < c1; w += NT) {
            const int u = w % w1 - 1, v = w / w1 - 1;
            const long long p = cell(u, v, kk);
            Vec3<Z> f;
            f.x = f.y = f.z = A::zero();
            Z s[6];
            for (int q = 0; q < 6; ++q) s[q] = A::zero();
            if (p >= 0) {
                Z o[6];
                for (int q = 0; q < 6; ++q) o[q] = A::ld_field(a.src[HXY + q], p);
                const HOut r = h_update(p, sE0[b0][v + 2][u + 2], sE0[b0][v + 2][u + 1], sE0[b0][v + 1][u + 2],
                                        sE0[b0 ^ 1][v + 2][u + 2], o);
                f = r.f;
                for (int q = 0; q < 6; ++q) s[q] = r.s[q];
            }
            sH1[bh][v + 1][u + 1] = f;
            if (u >= 0 && v >= 0 && u <= nix && v <= niy)
                for (int q = 0; q < 6; ++q) sH1s[bh][q][v][u] = s[q];
            // E^1(k-1) at the same cell if it lies in the E^1 region [-1, nix] x [-1, niy]
            if (u <= nix && v <= niy) {
                const long long pe = cell(u, v, km);
                Vec3<Z> g;
                g.x = g.y = g.z = A::zero();
                Z out[6];
                for (int q = 0; q < 6; ++q) out[q] = A::zero();
                if (pe >= 0 && k - 1 >= z0 - 1) {
                    Z o[6];
                    for (int q = 0; q < 6; ++q) o[q] = A::ld_field(a.src[EXY + q], pe);
                    // H^1 at k-1 lives in sH1[bh ^ 1]; at k it is f (beyond a Dirichlet top, zero)
                    e_update(pe, sH1[bh ^ 1][v + 1][u + 1], sH1[bh ^ 1][v + 1][u + 2], sH1[bh ^ 1][v + 2][u + 1], f,
                             o, out);
                    g.x = A::add(out[0], out[1]);
                    g.y = A::add(out[2], out[3]);
                    g.z = A::add(out[4], out[5]);
                }
                sE1[be][v + 1][u + 1] = g;
                if (u >= 0 && v >= 0 && u < nix && v < niy)
                    for (int q = 0; q < 6; ++q) sE1s[be][q][v][u] = out[q];
            }
        }
        __syncthreads();
        // ---- DE: H^2(k-1) on the H^2 region (stores the tile part), then
        //      E^2(k-2) at the same cell if it is a tile cell
        const int k2 = k - 1, k3 = k - 2;
        if (k2 >= z0) {
            const int kk2 = zin(k2);
            for (int w = threadIdx.x; w < c2; w += NT) {
                const int u = w % w2, v = w / w2;
                const long long p = cell(u, v, kk2);
                Vec3<Z> f;
                f.x = f.y = f.z = A::zero();
                if (p >= 0) {
                    Z o[6];
                    for (int q = 0; q < 6; ++q) o[q] = sH1s[bh ^ 1][q][v][u];
                    const HOut r = h_update(p, sE1[be][v + 1][u + 1], sE1[be][v + 1][u], sE1[be][v][u + 1],
                                            sE1[be ^ 1][v + 1][u + 1], o);
                    f = r.f;
                    if (u < nix && v < niy && k2 < z1) {
                        for (int q = 0; q < 6; ++q) A::st_field(a.dst[HXY + q], p, r.s[q]);
                        if (want_norm) {
                            const Vec3<Z> f1 = sH1[bh ^ 1][v + 1][u + 1];
                            A::acc_d3(acc_d, f.x, f1.x, f.y, f1.y, f.z, f1.z);
                            A::acc_n3(acc_x, f.x, f.y, f.z);
                        }
                    }
                }
                sH2[b2][v][u] = f;
                if (k3 >= z0 && k3 < z1 && u < nix && v < niy) {
                    const long long kk3 = zin(k3);
                    const long long pe = cell(u, v, (int)kk3);
                    Z o[6], out[6];
                    for (int q = 0; q < 6; ++q) o[q] = sE1s[be ^ 1][q][v][u];
                    e_update(pe, sH2[b2 ^ 1][v][u], sH2[b2 ^ 1][v][u + 1], sH2[b2 ^ 1][v + 1][u], f, o, out);
                    for (int q = 0; q < 6; ++q) A::st_field(a.dst[EXY + q], pe, out[q]);
                    if (want_norm) {
                        const Vec3<Z> f1 = sE1[be ^ 1][v + 1][u + 1];
                        const Z fx = A::add(out[0], out[1]), fy = A::add(out[2], out[3]), fz = A::add(out[4], out[5]);
                        A::acc_d3(acc_d, fx, f1.x, fy, f1.y, fz, f1.z);
                        A::acc_n3(acc_x, fx, fy, fz);
                    }
                }
            }
        }
        b0 ^= 1;
        bh ^= 1;
        be ^= 1;
        b2 ^= 1;
    }

    if (want_norm) {
        double sd = A::acc_value(acc_d), sx = A::acc_value(acc_x);
        for (int o = 16; o > 0; o >>= 1) {
            sd += __shfl_down_sync(0xffffffffu, sd, o);
            sx += __shfl_down_sync(0xffffffffu, sx, o);
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) { red[0][warp] = sd; red[1][warp] = sx; }
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
