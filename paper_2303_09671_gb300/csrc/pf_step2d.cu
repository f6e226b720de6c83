// pf_step2d.cu -- the fused explicit step for 2D grids (FP32 and FP64).
//
// The method and discretisation of pf_step.cu (the brackets of Eqs. cs_nonvar
// / cl_nonvar at faces, Eq. phasefield_nonvar at cells with the re-derived
// driving force, conservative (c, d) update, forward Euler), laid out like the
// 3D kernel of pf_step3d.cu without its z-march:
//   * a CTA owns a TX x TY tile; thread (tx, ty) owns the two cells (x, y) and
//     (x, y+1), y = y0 + 2 ty, evaluated as one two-lane vector (packed
//     .f32x2 arithmetic in FP32, see pf_lanes.cuh);
//   * the halo-2 tile is loaded once, converted to two-lane records
//     {phi, Y}, {mu_s, mu_l}, {c_s, c_l} and phi in shared memory; the rate
//     dx^2 dphi/dt is evaluated on the halo-1 ring (each thread its own pair,
//     the last warps the ring's border); each thread then evaluates the x+1/2
//     and y+1/2 faces of its pair (warps 0 and 1 also the tile's low edges) and
//     updates its two cells;
//   * the 9-point Laplacian is [4 faces, 1 corners, -20] / (6 dx^2), the
//     5-point one [1 faces, -4] / dx^2.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include "pf_internal.cuh"
#include "pf_kernels.h"
#include "pf_lanes.cuh"

namespace pf {

template <typename T, int TX, int TY>
struct PTile2 {
    static_assert(TY % 2 == 0, "cells are paired along y");
    using V = typename Lanes<T>::V;
    using Q = Q2<V>;
    static constexpr int TYP = TY / 2;                  // pair rows
    static constexpr int NT = TX * TYP;                 // threads
    static constexpr int HX = TX + 4, HYP = TYP + 2;    // halo-2 tile in pair cells
    static constexpr int HP = HX * HYP;
    static constexpr int RW = TX + 2, RX = HX;          // halo-1 ring (all pair rows), pitch HX
    static constexpr int NR = RW * HYP;
    static constexpr int JH = (HP + NT - 1) / NT;
    static constexpr int NB = NR - NT;                  // ring cells besides the own pairs
    static_assert(NB == 2 * RW + 2 * TYP && NB <= NT, "ring = own pairs + border");
    static constexpr size_t OFF_A = 0;                               // {phi, Y}
    static constexpr size_t OFF_B = OFF_A + sizeof(Q) * HP;          // {mu_s, mu_l}
    static constexpr size_t OFF_C = OFF_B + sizeof(Q) * HP;          // {c_s, c_l}
    static constexpr size_t OFF_P = OFF_C + sizeof(Q) * HP;          // phi
    static constexpr size_t OFF_D = OFF_P + sizeof(V) * HP;          // dx^2 phidot on the ring
    static constexpr size_t OFF_FX = OFF_D + sizeof(V) * HP;         // x faces {F_c, F_d}
    static constexpr size_t OFF_FY = OFF_FX + sizeof(Q) * TYP * (TX + 1);   // upper y face
    static constexpr size_t BYTES = OFF_FY + sizeof(V) * (TYP + 1) * TX;
};

template <typename T, int TX, int TY, bool L9, bool AI>
__global__ void __launch_bounds__(TX * (TY / 2), sizeof(T) == 4 ? 3 : 1)
step2d_kernel(const T* __restrict__ phi_in, const T* __restrict__ c_in, const T* __restrict__ d_in,
              const T* __restrict__ clo_in, T* __restrict__ phi_out, T* __restrict__ c_out,
              T* __restrict__ d_out, T* __restrict__ clo_out, const PairConsts<typename Lanes<T>::V> K,
              const GridConsts<T> G) {
    using L = PTile2<T, TX, TY>;
    using V = typename L::V;
    using Q = typename L::Q;
    constexpr int HX = L::HX, HP = L::HP, RX = L::RX, RW = L::RW, NT = L::NT, TYP = L::TYP, NB = L::NB;
    static_assert(HP < 4096, "tile too large for the packed ring descriptors");
    static_assert(NT >= 32 + TX && TYP <= 32, "edge faces need warps 0 and 1");
    extern __shared__ __align__(16) unsigned char smem[];
    Q* sA = reinterpret_cast<Q*>(smem + L::OFF_A);
    Q* sB = reinterpret_cast<Q*>(smem + L::OFF_B);
    Q* sC = reinterpret_cast<Q*>(smem + L::OFF_C);
    V* sP = reinterpret_cast<V*>(smem + L::OFF_P);
    V* sD = reinterpret_cast<V*>(smem + L::OFF_D);
    Q* sFx = reinterpret_cast<Q*>(smem + L::OFF_FX);
    V* sFy = reinterpret_cast<V*>(smem + L::OFF_FY);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nx = G.n[0], ny = G.n[1];
    const int own_h = (ty + 1) * HX + tx + 2;
    const int own_r = (ty + 1) * RX + tx + 1;
    const int own_x = x0 + tx, own_y = y0 + 2 * ty;
    const bool in_lo = own_x < nx && own_y < ny;
    const bool in_hi = own_x < nx && own_y + 1 < ny;
    const long long own_xy = (long long)own_y * nx + own_x;

    // own state for the update, in flight while the tile is converted
    T oc[2] = {T(0), T(0)}, od[2] = {T(0), T(0)}, olo[2] = {T(0), T(0)};
    if (in_lo) {
        oc[0] = c_in[own_xy];
        od[0] = d_in[own_xy];
        if (clo_in != nullptr) olo[0] = clo_in[own_xy];
    }
    if (in_hi) {
        oc[1] = c_in[own_xy + nx];
        od[1] = d_in[own_xy + nx];
        if (clo_in != nullptr) olo[1] = clo_in[own_xy + nx];
    }

    // ---- A: the halo-2 tile into two-lane records
#pragma unroll
    for (int j = 0; j < L::JH; ++j) {
        const int h = tid + j * NT;
        if ((j + 1) * NT > HP && h >= HP) break;
        const int mx = map_coord(x0 - 2 + h % HX, nx, G.bc_lo[0], G.bc_hi[0]);
        T f2[2], c2[2], d2[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int my = map_coord(y0 - 2 + 2 * (h / HX) + l, ny, G.bc_lo[1], G.bc_hi[1]);
            f2[l] = G.dir_phi;
            c2[l] = G.dir_c;
            d2[l] = G.dir_d;
            if (mx >= 0 && my >= 0) {
                const long long gi = (long long)my * nx + mx;
                f2[l] = phi_in[gi];
                c2[l] = c_in[gi];
                d2[l] = d_in[gi];
            }
        }
        const V f = vpair(f2[0], f2[1]), c = vpair(c2[0], c2[1]), d = vpair(d2[0], d2[1]);
        const V p = vp_of<AI>(K, f);
        const V cs = vfma(vsub(vlit<V>(1.0), p), d, c);
        const V cl = vsub(c, vmul(p, d));
        const V mus = vsub(vlog(cs), K.log_ke);
        const V mul = vlog(cl);
        sA[h] = Q{f, vfma(p, vsub(mus, mul), mul)};
        sB[h] = Q{mus, mul};
        sC[h] = Q{cs, cl};
        sP[h] = f;
    }
    __syncthreads();

    // ---- B: dx^2 phidot on the ring: the thread's own pair, and for the last
    // NB threads one border cell
    auto rate_cell = [&](int rx, int ry) {
        const int h = ry * HX + rx + 1;
        const int gxi = x0 - 1 + rx;
        const int mx = map_coord(gxi, nx, G.bc_lo[0], G.bc_hi[0]);
        const bool glo = mx < 0 || map_coord(y0 - 2 + 2 * ry, ny, G.bc_lo[1], G.bc_hi[1]) < 0;
        const bool ghi = mx < 0 || map_coord(y0 - 1 + 2 * ry, ny, G.bc_lo[1], G.bc_hi[1]) < 0;
        const int hS = (ry == 0) ? h : h - HX;              // first pair row: row below unused
        const int hN = (ry == L::HYP - 1) ? h : h + HX;     // last pair row: row above unused
        const T xc = (T((mx < 0) ? gxi : mx) + T(0.5)) * G.dx;   // theta at the mirror / wrap image
        const V f = sP[h];
        const V fxm = sP[h - 1], fxp = sP[h + 1], fS = sP[hS], fN = sP[hN];
        const V XP = vadd(fxm, fxp);
        const V faces = vadd(XP, vpair(fS.y + f.y, f.x + fN.x));
        V lap;
        if (L9) {
            const V XS = vadd(sP[hS - 1], sP[hS + 1]), XN = vadd(sP[hN - 1], sP[hN + 1]);
            const V corners = vpair(XS.y + XP.y, XP.x + XN.x);
            // [4 faces + corners - 20 centre] / 6
            lap = vmul(vlit<V>((1.0 / 6)), vfma(vlit<V>(4.0), vsub(faces, vfma(vlit<V>(4.0), f, f)), corners));
        } else {
            lap = vsub(faces, vmul(vlit<V>(4.0), f));
        }
        const Q cc = sC[h], bc = sB[h];
        const Q bxm = sB[h - 1], bxp = sB[h + 1], bS = sB[hS], bN = sB[hN];
        // centred differences (times 2 dx) of phi, mu_s, mu_l
        const V gx = vsub(fxp, fxm), gy = vpair(f.y - fS.y, fN.x - f.x);
        const V sx = vsub(bxp.a, bxm.a), sy = vpair(bc.a.y - bS.a.y, bN.a.x - bc.a.x);
        const V lx = vsub(bxp.b, bxm.b), ly = vpair(bc.b.y - bS.b.y, bN.b.x - bc.b.x);
        const V cs = cc.a, cl = cc.b, mus = bc.a, mul = bc.b;
        const V p = vp_of<AI>(K, f), dp = vdp_of<AI>(K, f);
        const V omp = vsub(vlit<V>(1.0), p);
        const V Ms = vfma(K.Ms_c, cs, K.Ms_0), Ml = vfma(K.Ml_c, cl, K.Ml_0);
        const V bMl = vmul(K.b, Ml);
        const V Msq = vmul(Ms, omp);
        const V iMbar = vrcp(vfma(bMl, p, Msq));
        const V d = vsub(cs, cl);
        const V g2 = vfma(gx, gx, vmul(gy, gy));
        const V cross = vsub(vmul(Ms, vfma(sx, gx, vmul(sy, gy))), vmul(bMl, vfma(lx, gx, vmul(ly, gy))));
        const V rr = vrcp(vadd(g2, K.delta2_4dx2));
        const V pq = vmul(p, omp);
        const V Kc = vfma(K.K_anti, vmul(vmul(vmul(d, d), vmul(pq, rr)), vmul(iMbar, vrcp(vfma(K.b, p, omp)))),
                          K.inv_Mphi);
        const T th_s = G.theta0 - G.G_theta * xc;
        const V theta = vpair(th_s, th_s);
        const V dmu = vsub(mus, mul);
        // D = [M_s (1-p)(1 - A(1-p)) + A b M_l p^2] / Mbar
        const V Dd = vmul(vfma(Msq, vsub(vlit<V>(1.0), vmul(K.A, omp)), vmul(vmul(K.A, bMl), vmul(p, p))), iMbar);
        // DeltaG = c_s (mu_s - mu_l) - d - (1-k_e) theta - D d (mu_s - mu_l)
        const V dG = vsub(vsub(vmul(cs, dmu), d), vfma(K.one_m_ke, theta, vmul(vmul(Dd, d), dmu)));
        const V g = vmul(f, vsub(vlit<V>(1.0), f));
        const V dfdw = vmul(g, vsub(vlit<V>(2.0), vmul(vlit<V>(4.0), f)));
        const V anti = vmul(vmul(vmul(K.one_m_A, d), vmul(pq, iMbar)), vmul(cross, rr));
        const V R = vfma(K.sigma, lap, vmul(K.dx2, vsub(anti, vfma(K.H, dfdw, vmul(dG, dp)))));
        sD[ry * RX + rx] = vmask(vmul(R, vrcp(Kc)), glo, ghi);
    };
    rate_cell(tx + 1, ty + 1);
    if (tid >= NT - NB) {
        const int b = tid - (NT - NB);
        if (b < RW) rate_cell(b, 0);
        else if (b < 2 * RW) rate_cell(b - RW, L::HYP - 1);
        else if (b < 2 * RW + TYP) rate_cell(0, 1 + b - 2 * RW);
        else rate_cell(RW - 1, 1 + b - 2 * RW - TYP);
    }
    __syncthreads();

    // ---- C: faces.  Components 0..3 = phi, Y, mu_s, mu_l = (A.a, A.b, B.a, B.b).
    // x face between halo cells hL and hL + 1 (ring index rL of hL)
    auto xface = [&](int hL, int rL, V& Fc, V& Fd) {
        const int hR = hL + 1;
        const Q aL = sA[hL], aR = sA[hR], bL = sB[hL], bR = sB[hR];
        V n[4] = {vsub(aR.a, aL.a), vsub(aR.b, aL.b), vsub(bR.a, bL.a), vsub(bR.b, bL.b)};
        // y: the rows of a pair are its two lanes
        const Q aS = sA[hL - HX], aS1 = sA[hR - HX], aN = sA[hL + HX], aN1 = sA[hR + HX];
        const Q bS = sB[hL - HX], bS1 = sB[hR - HX], bN = sB[hL + HX], bN1 = sB[hR + HX];
        V SP[4] = {vadd(aL.a, aR.a), vadd(aL.b, aR.b), vadd(bL.a, bR.a), vadd(bL.b, bR.b)};
        V SS[4] = {vadd(aS.a, aS1.a), vadd(aS.b, aS1.b), vadd(bS.a, bS1.a), vadd(bS.b, bS1.b)};
        V SN[4] = {vadd(aN.a, aN1.a), vadd(aN.b, aN1.b), vadd(bN.a, bN1.a), vadd(bN.b, bN1.b)};
        V t1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) t1[k] = vpair(SP[k].y - SS[k].y, SN[k].x - SP[k].x);
        const Q cL = sC[hL], cR = sC[hR];
        face_flux<V, false, AI>(K, vmul(vlit<V>(0.5), SP[0]), vadd(cL.a, cR.a), vadd(cL.b, cR.b),
                            vadd(sD[rL], sD[rL + 1]), n, t1, t1, Fc, Fd);
    };
    // y faces above the two rows of the pair at hL: lanes (y+1/2, y+3/2)
    auto yface = [&](int hL, int rL, V& Fc, V& Fd) {
        const int hN = hL + HX;
        const Q aP = sA[hL], aN = sA[hN], bP = sB[hL], bN = sB[hN];
        const V cP[4] = {aP.a, aP.b, bP.a, bP.b};
        const V cN[4] = {aN.a, aN.b, bN.a, bN.b};
        V n[4], t1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) n[k] = vpair(cP[k].y - cP[k].x, cN[k].x - cP[k].y);
        // x: differences at both pairs, then the two rows of each face
        const Q aPp = sA[hL + 1], aPm = sA[hL - 1], aNp = sA[hN + 1], aNm = sA[hN - 1];
        const Q bPp = sB[hL + 1], bPm = sB[hL - 1], bNp = sB[hN + 1], bNm = sB[hN - 1];
        const V DP[4] = {vsub(aPp.a, aPm.a), vsub(aPp.b, aPm.b), vsub(bPp.a, bPm.a), vsub(bPp.b, bPm.b)};
        const V DN[4] = {vsub(aNp.a, aNm.a), vsub(aNp.b, aNm.b), vsub(bNp.a, bNm.a), vsub(bNp.b, bNm.b)};
#pragma unroll
        for (int k = 0; k < 4; ++k) t1[k] = vpair(DP[k].x + DP[k].y, DP[k].y + DN[k].x);
        const Q cP_ = sC[hL], cN_ = sC[hN];
        const V dP = sD[rL], dN = sD[rL + RX];
        const V f = vmul(vlit<V>(0.5), vpair(cP[0].x + cP[0].y, cP[0].y + cN[0].x));
        const V cs2 = vpair(cP_.a.x + cP_.a.y, cP_.a.y + cN_.a.x);
        const V cl2 = vpair(cP_.b.x + cP_.b.y, cP_.b.y + cN_.b.x);
        face_flux<V, false, AI>(K, f, cs2, cl2, vpair(dP.x + dP.y, dP.y + dN.x), n, t1, t1, Fc, Fd);
    };
    const bool nf_x = own_x == nx - 1 && G.bc_hi[0] == BC_NOFLUX;
    const bool nf_ylo = own_y == ny - 1 && G.bc_hi[1] == BC_NOFLUX;
    const bool nf_yhi = own_y + 1 == ny - 1 && G.bc_hi[1] == BC_NOFLUX;
    V fxc, fxd, fyc, fyd;
    xface(own_h, own_r, fxc, fxd);
    yface(own_h, own_r, fyc, fyd);
    if (nf_x) fxc = fxd = vpair(T(0), T(0));
    fyc = vmask(fyc, nf_ylo, nf_yhi);
    fyd = vmask(fyd, nf_ylo, nf_yhi);
    sFx[ty * (TX + 1) + tx + 1] = Q{fxc, fxd};
    sFy[(ty + 1) * TX + tx] = vpair(fyc.y, fyd.y);
    if (tid < TYP) {
        // x faces on the tile's low x edge, pair row tid
        V ec, ed;
        xface((tid + 1) * HX + 1, (tid + 1) * RX, ec, ed);
        if (x0 == 0 && G.bc_lo[0] == BC_NOFLUX) ec = ed = vpair(T(0), T(0));
        sFx[tid * (TX + 1)] = Q{ec, ed};
    } else if (tid >= 32 && tid < 32 + TX) {
        // y face on the tile's low y edge (upper lane of the pair row below the tile)
        const int ex = tid - 32;
        V ec, ed;
        yface(ex + 2, ex + 1, ec, ed);
        sFy[ex] = (y0 == 0 && G.bc_lo[1] == BC_NOFLUX) ? vpair(T(0), T(0)) : vpair(ec.y, ed.y);
    }
    __syncthreads();

    // ---- D: conservative update of the pair
    const Q left = sFx[ty * (TX + 1) + tx];
    const V below = sFy[ty * TX + tx];
    const V dFc = vadd(vsub(fxc, left.a), vpair(fyc.x - below.x, fyc.y - fyc.x));
    const V dFd = vadd(vsub(fxd, left.b), vpair(fyd.x - below.y, fyd.y - fyd.x));
    const V c_k = vpair(oc[0], oc[1]), d_k = vpair(od[0], od[1]);
    const V phi_new = vfma(K.dt_dx2, sD[own_r], sA[own_h].a);
    const V d_new = vfma(K.dt_dx2, dFd, d_k);
    const V dcv = vmul(K.dt_dx2, dFc);
    V c_new, lo_new;
    if (clo_in != nullptr) {
        // compensated (TwoSum) update of c = hi + lo
        const V lo_k = vpair(olo[0], olo[1]);
        const V s_ = vadd(c_k, dcv);
        const V bv = vsub(s_, c_k);
        const V err = vadd(vsub(c_k, vsub(s_, bv)), vsub(dcv, bv));
        const V lo = vadd(lo_k, err);
        c_new = vadd(s_, lo);
        lo_new = vsub(lo, vsub(c_new, s_));
    } else {
        c_new = vadd(c_k, dcv);
        lo_new = c_new;
    }
    if (in_lo) {
        phi_out[own_xy] = phi_new.x;
        c_out[own_xy] = c_new.x;
        d_out[own_xy] = d_new.x;
        if (clo_out != nullptr) clo_out[own_xy] = lo_new.x;
    }
    if (in_hi) {
        phi_out[own_xy + nx] = phi_new.y;
        c_out[own_xy + nx] = c_new.y;
        d_out[own_xy + nx] = d_new.y;
        if (clo_out != nullptr) clo_out[own_xy + nx] = lo_new.y;
    }
}

template <typename T>
cudaError_t launch_step2d(const StepLaunch& a, const Consts<T>& C, const Clock<T>& Kc) {
    constexpr int TX = 32, TY = 16;
    using L = PTile2<T, TX, TY>;
    // 9- or 5-point Laplacian x shape parameter a != 0 or a = 0
    decltype(&step2d_kernel<T, TX, TY, true, true>) kerns[2][2] = {
        {step2d_kernel<T, TX, TY, false, false>, step2d_kernel<T, TX, TY, false, true>},
        {step2d_kernel<T, TX, TY, true, false>, step2d_kernel<T, TX, TY, true, true>}};
    static DeviceSetup setup;
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= DeviceSetup::MAX_DEVICES) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lock(setup.mu);
        if (!setup.done[dev]) {
            for (int i = 0; i < 4 && e == cudaSuccess; ++i)
                e = cudaFuncSetAttribute(kerns[i / 2][i % 2], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L::BYTES);
            if (e != cudaSuccess) return e;
            setup.done[dev] = true;
        }
    }
    const HostProblem& P = *a.prob;
    const PairConsts<typename L::V> K = make_pair_consts<T>(P, C);
    const GridConsts<T> G = make_grid_consts<T>(P, Kc);
    const dim3 block(L::NT);
    const dim3 grid((C.n[0] + TX - 1) / TX, (C.n[1] + TY - 1) / TY, 1);
    auto kern = kerns[C.lap == 9 ? 1 : 0][P.a != 0.0 ? 1 : 0];
    kern<<<grid, block, L::BYTES, a.stream>>>(
        static_cast<const T*>(a.phi_in), static_cast<const T*>(a.c_in), static_cast<const T*>(a.d_in),
        static_cast<const T*>(a.clo_in), static_cast<T*>(a.phi_out), static_cast<T*>(a.c_out),
        static_cast<T*>(a.d_out), static_cast<T*>(a.clo_out), K, G);
    return cudaGetLastError();
}

template cudaError_t launch_step2d<float>(const StepLaunch&, const Consts<float>&, const Clock<float>&);
template cudaError_t launch_step2d<double>(const StepLaunch&, const Consts<double>&, const Clock<double>&);

}  // namespace pf
