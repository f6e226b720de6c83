// pf_step.cu -- the fused explicit time step (one kernel per step).
//
// One CTA owns a TX x TY tile of columns and marches along z (2.5D): each
// z-plane of phi, c_s, c_l is read from HBM once (with a 2-cell xy halo, kept
// in a 4-slot shared-memory ring), and each output plane is written once.
// Per plane k the pipeline is
//   A  load plane k+2 (halo 2) and its pointwise values mu_s, mu_l, Y
//   B  plane k+1 on the ring-1 region: centred gradients of phi, Y, mu_s, mu_l
//      and the phase-field rate (Eq. phasefield_nonvar, re-derived DeltaG)
//   C  the face fluxes of plane k (x and y faces in shared memory, the z face
//      to plane k+1 in registers): brackets of Eqs. cs_nonvar / cl_nonvar,
//      combined into F_c = p_f F_s + (1-p_f) F_l and F_d = F_s - F_l
//   D  conservative update of c and d, Euler update of phi (Sec. "Numerical
//      technique").  The state is held as (phi, c, d) with c = p c_s + (1-p) c_l
//      (Eq. model1) and d = c_s - c_l; c_s = c + (1-p) d and c_l = c - p d are
//      rebuilt from it when a plane is loaded.  In FP32, c carries a second
//      FP32 word (compensated sum) so that its conservative update loses no
//      solute to rounding.
// 2D and 1D grids use the same kernel with one plane (and one row).
#include <cstdint>
#include <cstdio>
#include <cmath>
#include <algorithm>
#include "pf_internal.cuh"
#include "pf_kernels.h"

namespace pf {

template <typename T, int DIM, int TX, int TY>
struct Tile {
    static constexpr int TYe = (DIM >= 2) ? TY : 1;
    static constexpr int HX = TX + 4;
    static constexpr int HY = (DIM >= 2) ? TY + 4 : 1;
    static constexpr int RX = TX + 2;
    static constexpr int RY = (DIM >= 2) ? TY + 2 : 1;
    static constexpr int NS = (DIM == 3) ? 4 : 1;   // raw/pointwise plane slots
    static constexpr int NG = (DIM == 3) ? 2 : 1;   // gradient / rate plane slots
    static constexpr int HP = HX * HY;               // halo-2 plane size
    static constexpr int RP = RX * RY;               // ring-1 plane size
    static constexpr int NFX = (TX + 1) * TYe;
    static constexpr int NFY = (DIM >= 2) ? TX * (TY + 1) : 0;
    // shared-memory layout, in units of T
    static constexpr int OFF_RAW = 0;                             // [6][NS][HP]: phi cs cl mus mul Y
    static constexpr int OFF_G = OFF_RAW + 6 * NS * HP;            // [4*DIM][NG][RP]
    static constexpr int OFF_PD = OFF_G + 4 * DIM * NG * RP;       // [NG][RP]
    static constexpr int OFF_FX = OFF_PD + NG * RP;                // [2][NFX]
    static constexpr int OFF_FY = OFF_FX + 2 * NFX;                // [2][NFY]
    static constexpr int TOTAL = OFF_FY + 2 * NFY;
    static constexpr size_t BYTES = sizeof(T) * (size_t)TOTAL;
};

// Face fluxes between cells L and R along `axis`.  Normal components of the
// face gradients are one-sided differences, the transverse ones the means of
// the two cells' centred differences; phi, c_s, c_l, d and phidot at the face
// are the means of the two cells; p, Mbar, q_n and the weights are evaluated
// at the face phi.
template <typename T>
cudaError_t launch_step3d(const StepLaunch& a, const Consts<T>& C, const Clock<T>& K);
template <typename T>
cudaError_t launch_step2d(const StepLaunch& a, const Consts<T>& C, const Clock<T>& K);

template <typename T, int DIM>
__device__ __forceinline__ void face_flux(const Consts<T>& C, int axis,
                                          T phiL, T phiR, T csL, T csR, T clL, T clR,
                                          T pdL, T pdR, const T nrm[4],
                                          const T trn[4][3], T& Fc, T& Fd) {
    const T f = T(0.5) * (phiL + phiR);
    const T cs = T(0.5) * (csL + csR);
    const T cl = T(0.5) * (clL + clR);
    const T d = cs - cl;
    const T pdot = T(0.5) * (pdL + pdR);
    const T p = p_of(C, f);
    const T Ms = Ms_of(C, cs), Ml = Ml_of(C, cl);
    const T bMlp = C.b * Ml * p;
    const T Mbar = Ms * (T(1) - p) + bMlp;
    const T iMbar = T(1) / Mbar;
    const T q = Ms * Ml * (C.b * p + T(1) - p) * iMbar;
    const T ws = Ms * (T(1) - p) * iMbar;
    const T wl = bMlp * iMbar;
    // gradient vectors of phi, Y, mu_s, mu_l at the face: normal component
    // nrm[.], transverse components trn[.][e]
    T gt2 = T(0), dYt = T(0), dst = T(0), dlt = T(0);
#pragma unroll
    for (int e = 0; e < DIM - 1; ++e) {
        gt2 += trn[0][e] * trn[0][e];
        dYt += trn[0][e] * trn[1][e];
        dst += trn[0][e] * trn[2][e];
        dlt += trn[0][e] * trn[3][e];
    }
    const T ga = nrm[0];
    const T gt2d = gt2 + C.delta2;
    const T r = T(1) / (ga * ga + gt2d);
    const T dY = ga * nrm[1] + dYt;
    const T normal = q * ga * dY * r;
    const T at = C.one_m_A * d * pdot * ga * r;
    // tangential part d_a mu - g_a (g.grad mu) r, rewritten without cancellation
    // as [d_a mu (|g_t|^2 + delta^2) - g_a (g_t.grad_t mu)] r
    const T Fs = normal + Ms * (nrm[2] * gt2d - ga * dst) * r + at * ws;
    const T Fl = normal + Ml * (nrm[3] * gt2d - ga * dlt) * r - at * wl;
    Fc = p * Fs + (T(1) - p) * Fl;
    Fd = Fs - Fl;
    (void)axis;
}

template <typename T, int DIM, int TX, int TY>
__global__ void __launch_bounds__(TX *(DIM >= 2 ? TY : 1))
step_kernel(const T* __restrict__ phi_in, const T* __restrict__ c_in,
            const T* __restrict__ d_in, const T* __restrict__ clo_in, const T* __restrict__ plo_in,
            T* __restrict__ phi_out, T* __restrict__ c_out, T* __restrict__ d_out,
            T* __restrict__ clo_out, T* __restrict__ plo_out, Consts<T> C, Clock<T> K, int zchunk) {
    using L = Tile<T, DIM, TX, TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* sRaw = sm + L::OFF_RAW;
    T* sG = sm + L::OFF_G;
    T* sPd = sm + L::OFF_PD;
    T* sFx = sm + L::OFF_FX;
    T* sFy = sm + L::OFF_FY;

    const int nthreads = TX * L::TYe;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX;
    const int y0 = (DIM >= 2) ? blockIdx.y * TY : 0;
    const int nx = C.n[0], ny = C.n[1], nz = C.n[2];
    const long long sy = nx, sz = (long long)nx * ny;

    auto RAW = [&](int field, int slot, int h) -> T& {
        return sRaw[(field * L::NS + slot) * L::HP + h];
    };
    auto GR = [&](int comp, int slot, int r) -> T& {   // comp = field*DIM + axis
        return sG[(comp * L::NG + slot) * L::RP + r];
    };
    auto PD = [&](int slot, int r) -> T& { return sPd[slot * L::RP + r]; };

    // ---- A: load plane z (halo 2) into slot s with its pointwise values
    auto load_plane = [&](int z, int s) {
        int mz = 0;
        bool dirz = false;
        if constexpr (DIM == 3) {
            mz = map_coord(z, nz, C.bc_lo[2], C.bc_hi[2]);
            dirz = (mz == DIR_GHOST);
        }
        for (int h = tid; h < L::HP; h += nthreads) {
            const int hx = h % L::HX, hy = h / L::HX;
            const int gx = x0 - 2 + hx;
            const int mx = map_coord(gx, nx, C.bc_lo[0], C.bc_hi[0]);
            int my = 0;
            bool dir = dirz || (mx < 0);
            if constexpr (DIM >= 2) {
                my = map_coord(y0 - 2 + hy, ny, C.bc_lo[1], C.bc_hi[1]);
                dir = dir || (my < 0);
            }
            T f, cs, cl, p;
            if (dir) {
                f = C.dir_phi; cs = C.dir_cs; cl = C.dir_cl;
                p = p_of(C, f);
            } else {
                const long long gi = (long long)mz * sz + (long long)my * sy + mx;
                f = phi_in[gi];
                const T c = c_in[gi], d = d_in[gi];
                p = p_of(C, f);
                cs = c + (T(1) - p) * d;   // c_s, c_l from c = p c_s + (1-p) c_l, d = c_s - c_l
                cl = c - p * d;
            }
            const T mus = flog(cs) - C.log_ke;
            const T mul = flog(cl);
            RAW(0, s, h) = f;
            RAW(1, s, h) = cs;
            RAW(2, s, h) = cl;
            RAW(3, s, h) = mus;
            RAW(4, s, h) = mul;
            RAW(5, s, h) = p * mus + (T(1) - p) * mul;
        }
    };

    // ---- B: centred gradients and phase-field rate of plane z on the ring-1 region
    // slots: sm = slot of plane z-1, s0 = plane z, sp = plane z+1; g = gradient slot
    auto rates_plane = [&](int z, int sM, int s0, int sP, int g) {
        const T theta_base = K.theta0;
        bool dirz = false;
        if constexpr (DIM == 3) dirz = (map_coord(z, nz, C.bc_lo[2], C.bc_hi[2]) == DIR_GHOST);
        for (int r = tid; r < L::RP; r += nthreads) {
            const int rx = r % L::RX, ry = r / L::RX;
            const int hx = rx + 1, hy = (DIM >= 2) ? ry + 1 : 0;
            const int h = hy * L::HX + hx;
            const int gx = x0 - 1 + rx;
            const int mx = map_coord(gx, nx, C.bc_lo[0], C.bc_hi[0]);
            bool dir = dirz || (mx < 0);
            if constexpr (DIM >= 2) dir = dir || (map_coord(y0 - 1 + ry, ny, C.bc_lo[1], C.bc_hi[1]) < 0);
            // centred gradients of phi, Y, mu_s, mu_l
            T gr[4][3];
            const int fld[4] = {0, 5, 3, 4};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                gr[q][0] = (RAW(fld[q], s0, h + 1) - RAW(fld[q], s0, h - 1)) * C.inv_2dx;
                if constexpr (DIM >= 2)
                    gr[q][1] = (RAW(fld[q], s0, h + L::HX) - RAW(fld[q], s0, h - L::HX)) * C.inv_2dx;
                if constexpr (DIM == 3)
                    gr[q][2] = (RAW(fld[q], sP, h) - RAW(fld[q], sM, h)) * C.inv_2dx;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int e = 0; e < DIM; ++e) GR(q * DIM + e, g, r) = gr[q][e];
            // Laplacian
            const T fc = RAW(0, s0, h);
            T lap;
            if constexpr (DIM == 1) {
                lap = (RAW(0, s0, h - 1) - fc) + (RAW(0, s0, h + 1) - fc);
            } else if constexpr (DIM == 2) {
                const T fE = RAW(0, s0, h + 1) - fc, fW = RAW(0, s0, h - 1) - fc;
                const T fN = RAW(0, s0, h + L::HX) - fc, fS = RAW(0, s0, h - L::HX) - fc;
                if (C.lap == 5) {
                    lap = fW + fE + fS + fN;
                } else {
                    const T cNE = RAW(0, s0, h + L::HX + 1) - fc, cNW = RAW(0, s0, h + L::HX - 1) - fc;
                    const T cSE = RAW(0, s0, h - L::HX + 1) - fc, cSW = RAW(0, s0, h - L::HX - 1) - fc;
                    lap = T(2.0 / 3.0) * (fW + fE + fS + fN) + T(1.0 / 6.0) * (cSW + cSE + cNW + cNE);
                }
            } else {
                const T fE = RAW(0, s0, h + 1) - fc, fW = RAW(0, s0, h - 1) - fc;
                const T fN = RAW(0, s0, h + L::HX) - fc, fS = RAW(0, s0, h - L::HX) - fc;
                const T fU = RAW(0, sP, h) - fc, fD = RAW(0, sM, h) - fc;
                if (C.lap == 7) {
                    lap = fW + fE + fS + fN + fD + fU;
                } else {
                    const T e_xy = (RAW(0, s0, h + L::HX + 1) - fc) + (RAW(0, s0, h + L::HX - 1) - fc) +
                                   (RAW(0, s0, h - L::HX + 1) - fc) + (RAW(0, s0, h - L::HX - 1) - fc);
                    const T e_xz = (RAW(0, sP, h + 1) - fc) + (RAW(0, sP, h - 1) - fc) +
                                   (RAW(0, sM, h + 1) - fc) + (RAW(0, sM, h - 1) - fc);
                    const T e_yz = (RAW(0, sP, h + L::HX) - fc) + (RAW(0, sP, h - L::HX) - fc) +
                                   (RAW(0, sM, h + L::HX) - fc) + (RAW(0, sM, h - L::HX) - fc);
                    lap = T(1.0 / 3.0) * (fW + fE + fS + fN + fD + fU) + T(1.0 / 6.0) * (e_xy + e_xz + e_yz);
                }
            }
            lap *= C.inv_dx2;
            // phase-field rate
            T pd;
            if (dir) {
                pd = T(0);
            } else {
                const T cs = RAW(1, s0, h), cl = RAW(2, s0, h);
                const T mus = RAW(3, s0, h), mul = RAW(4, s0, h);
                const T p = p_of(C, fc), dp = dp_of(C, fc);
                const T Ms = Ms_of(C, cs), Ml = Ml_of(C, cl);
                const T bMl = C.b * Ml;
                const T Mbar = Ms * (T(1) - p) + bMl * p;
                const T iMbar = T(1) / Mbar;
                const T d = cs - cl;
                T g2 = T(0), cross = T(0);
#pragma unroll
                for (int e = 0; e < DIM; ++e) {
                    g2 += gr[0][e] * gr[0][e];
                    cross += (Ms * gr[2][e] - bMl * gr[3][e]) * gr[0][e];
                }
                const T rr = T(1) / (g2 + C.delta2);
                const T pq = p * (T(1) - p);
                const T Kc = C.inv_Mphi + C.one_m_A * C.one_m_A * d * d * C.b * pq * rr * iMbar /
                                              (C.b * p + T(1) - p);
                // theta at the (mapped) cell centre along x
                const int ix = (mx < 0) ? gx : mx;
                const T theta = theta_base - C.G_theta * ((T(ix) + T(0.5)) * C.dx);
                const T fs = -C.one_m_ke * theta + cs * (mus - T(1));
                const T fl = cl * (mul - T(1));
                const T D = (Ms * (T(1) - p) * (T(1) - C.A * (T(1) - p)) + C.A * bMl * p * p) * iMbar;
                const T dG = fs - fl - mul * d - D * d * (mus - mul);
                const T dfdw = T(2) * fc * (T(1) - fc) * (T(1) - T(2) * fc);
                const T R = C.sigma * lap - C.H * dfdw - dG * dp + C.one_m_A * d * pq * iMbar * cross * rr;
                pd = R / Kc;
            }
            PD(g, r) = pd;
        }
    };

    // z face between plane z (slots s0, g0) and z+1 (s1, g1) for this thread's column
    auto zface = [&](int z, int s0, int s1, int g0, int g1, T& Fc, T& Fd) {
        Fc = T(0); Fd = T(0);
        if constexpr (DIM != 3) { return; } else {
        const bool noflux = (z == -1 && C.bc_lo[2] == BC_NOFLUX) ||
                            (z == nz - 1 && C.bc_hi[2] == BC_NOFLUX);
        if (noflux) return;
        const int h = (ty + 2) * L::HX + (tx + 2);
        const int r = (ty + 1) * L::RX + (tx + 1);
        T nrm[4], trn[4][3];
        const int fld[4] = {0, 5, 3, 4};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            nrm[q] = (RAW(fld[q], s1, h) - RAW(fld[q], s0, h)) * C.inv_dx;
            trn[q][0] = T(0.5) * (GR(q * DIM + 0, g0, r) + GR(q * DIM + 0, g1, r));
            trn[q][1] = T(0.5) * (GR(q * DIM + 1, g0, r) + GR(q * DIM + 1, g1, r));
        }
        face_flux<T, DIM>(C, 2, RAW(0, s0, h), RAW(0, s1, h), RAW(1, s0, h), RAW(1, s1, h),
                          RAW(2, s0, h), RAW(2, s1, h), PD(g0, r), PD(g1, r), nrm, trn, Fc, Fd);
        }
    };

    // ---- C: x and y faces of plane z (slot s0, gradient slot g0) into shared memory
    auto xy_faces = [&](int s0, int g0) {
        const int fld[4] = {0, 5, 3, 4};
        for (int f = tid; f < L::NFX; f += nthreads) {
            const int fx = f % (TX + 1), fy = f / (TX + 1);
            const int gxl = x0 + fx - 1;   // left cell of the face
            T Fc = T(0), Fd = T(0);
            const bool noflux = (gxl == -1 && C.bc_lo[0] == BC_NOFLUX) ||
                                (gxl == nx - 1 && C.bc_hi[0] == BC_NOFLUX);
            if (!noflux) {
                const int hL = ((DIM >= 2) ? (fy + 2) : 0) * L::HX + (fx + 1);
                const int rL = ((DIM >= 2) ? (fy + 1) : 0) * L::RX + fx;
                T nrm[4], trn[4][3];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    nrm[q] = (RAW(fld[q], s0, hL + 1) - RAW(fld[q], s0, hL)) * C.inv_dx;
#pragma unroll
                    for (int e = 1; e < DIM; ++e)
                        trn[q][e - 1] = T(0.5) * (GR(q * DIM + e, g0, rL) + GR(q * DIM + e, g0, rL + 1));
                }
                face_flux<T, DIM>(C, 0, RAW(0, s0, hL), RAW(0, s0, hL + 1), RAW(1, s0, hL),
                                  RAW(1, s0, hL + 1), RAW(2, s0, hL), RAW(2, s0, hL + 1),
                                  PD(g0, rL), PD(g0, rL + 1), nrm, trn, Fc, Fd);
            }
            sFx[f] = Fc;
            sFx[L::NFX + f] = Fd;
        }
        if constexpr (DIM >= 2) {
            for (int f = tid; f < L::NFY; f += nthreads) {
                const int fx = f % TX, fy = f / TX;   // face below row fy (between fy-1 and fy)
                const int gyl = y0 + fy - 1;
                T Fc = T(0), Fd = T(0);
                const bool noflux = (gyl == -1 && C.bc_lo[1] == BC_NOFLUX) ||
                                    (gyl == ny - 1 && C.bc_hi[1] == BC_NOFLUX);
                if (!noflux) {
                    const int hL = (fy + 1) * L::HX + (fx + 2);
                    const int rL = fy * L::RX + (fx + 1);
                    T nrm[4], trn[4][3];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        nrm[q] = (RAW(fld[q], s0, hL + L::HX) - RAW(fld[q], s0, hL)) * C.inv_dx;
                        trn[q][0] = T(0.5) * (GR(q * DIM + 0, g0, rL) + GR(q * DIM + 0, g0, rL + L::RX));
                        if constexpr (DIM == 3)
                            trn[q][1] = T(0.5) * (GR(q * DIM + 2, g0, rL) + GR(q * DIM + 2, g0, rL + L::RX));
                    }
                    face_flux<T, DIM>(C, 1, RAW(0, s0, hL), RAW(0, s0, hL + L::HX), RAW(1, s0, hL),
                                      RAW(1, s0, hL + L::HX), RAW(2, s0, hL), RAW(2, s0, hL + L::HX),
                                      PD(g0, rL), PD(g0, rL + L::RX), nrm, trn, Fc, Fd);
                }
                sFy[f] = Fc;
                sFy[L::NFY + f] = Fd;
            }
        }
    };

    // ---- D: update of this thread's cell in plane z
    auto update = [&](int z, int s0, int g0, T FzcD, T FzdD, T FzcU, T FzdU) {
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx >= nx || (DIM >= 2 && gy >= ny) || z >= nz) return;
        const int h = ((DIM >= 2) ? (ty + 2) : 0) * L::HX + (tx + 2);
        const int r = ((DIM >= 2) ? (ty + 1) : 0) * L::RX + (tx + 1);
        T dc = sFx[ty * (TX + 1) + tx + 1] - sFx[ty * (TX + 1) + tx];
        T dd = sFx[L::NFX + ty * (TX + 1) + tx + 1] - sFx[L::NFX + ty * (TX + 1) + tx];
        if constexpr (DIM >= 2) {
            dc += sFy[(ty + 1) * TX + tx] - sFy[ty * TX + tx];
            dd += sFy[L::NFY + (ty + 1) * TX + tx] - sFy[L::NFY + ty * TX + tx];
        }
        if constexpr (DIM == 3) {
            dc += FzcU - FzcD;
            dd += FzdU - FzdD;
        }
        const long long gi = (long long)z * sz + (long long)gy * sy + gx;
        const T f = RAW(0, s0, h);
        const T dcv = C.dt * dc * C.inv_dx;
        if (plo_in != nullptr) {
            // phi = hi + lo, the increment added by TwoSum as for c below
            const T dp = C.dt * PD(g0, r);
            const T s = f + dp;
            const T bv = s - f;
            const T lo = plo_in[gi] + ((f - (s - bv)) + (dp - bv));
            const T hi = s + lo;
            phi_out[gi] = hi;
            plo_out[gi] = lo - (hi - s);
        } else {
            phi_out[gi] = f + C.dt * PD(g0, r);
        }
        d_out[gi] = d_in[gi] + C.dt * dd * C.inv_dx;
        const T c = c_in[gi];
        if (clo_in != nullptr) {
            // c held as an unevaluated sum hi + lo of two FP32 numbers; the
            // increment is added with an error-free transformation (Knuth's
            // TwoSum) so that total solute is conserved to ~FP64 accuracy
            const T s = c + dcv;
            const T bv = s - c;
            const T err = (c - (s - bv)) + (dcv - bv);
            const T lo = clo_in[gi] + err;
            const T hi = s + lo;
            c_out[gi] = hi;
            clo_out[gi] = lo - (hi - s);
        } else {
            c_out[gi] = c + dcv;
        }
    };

    if constexpr (DIM < 3) {
        load_plane(0, 0);
        __syncthreads();
        rates_plane(0, 0, 0, 0, 0);
        __syncthreads();
        xy_faces(0, 0);
        __syncthreads();
        update(0, 0, 0, T(0), T(0), T(0), T(0));
        return;
    } else {

    // ---- 3D z-march over the chunk [z0, z1)
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(nz, z0 + zchunk);
    if (z0 >= z1) return;
    // prologue: planes z0-2 .. z0+1, rates of z0-1 and z0, z face (z0-1, z0)
    for (int z = z0 - 2; z <= z0 + 1; ++z) load_plane(z, z & 3);
    __syncthreads();
    rates_plane(z0 - 1, (z0 - 2) & 3, (z0 - 1) & 3, z0 & 3, (z0 - 1) & 1);
    rates_plane(z0, (z0 - 1) & 3, z0 & 3, (z0 + 1) & 3, z0 & 1);
    __syncthreads();
    T FzcD, FzdD;
    zface(z0 - 1, (z0 - 1) & 3, z0 & 3, (z0 - 1) & 1, z0 & 1, FzcD, FzdD);
    for (int k = z0; k < z1; ++k) {
        load_plane(k + 2, (k + 2) & 3);
        __syncthreads();
        rates_plane(k + 1, k & 3, (k + 1) & 3, (k + 2) & 3, (k + 1) & 1);
        __syncthreads();
        xy_faces(k & 3, k & 1);
        T FzcU, FzdU;
        zface(k, k & 3, (k + 1) & 3, k & 1, (k + 1) & 1, FzcU, FzdU);
        __syncthreads();
        update(k, k & 3, k & 1, FzcD, FzdD, FzcU, FzdU);
        FzcD = FzcU;
        FzdD = FzdU;
    }
    }
}

// ------------------------------------------------------------------ launchers

template <typename T, int DIM, int TX, int TY>
static cudaError_t launch_tile(const StepLaunch& a, const Consts<T>& C, const Clock<T>& K) {
    using L = Tile<T, DIM, TX, TY>;
    auto kern = step_kernel<T, DIM, TX, TY>;
    static DeviceSetup setup;
    int dev = 0, per_sm = 1, sms = 1;
    {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= DeviceSetup::MAX_DEVICES) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lock(setup.mu);
        if (!setup.done[dev]) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
            if (e != cudaSuccess) return e;
            int s = 1, p = 1;
            cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, kern, TX * L::TYe, L::BYTES);
            setup.sms[dev] = s;
            setup.per_sm[dev] = p < 1 ? 1 : p;
            setup.done[dev] = true;
        }
        per_sm = setup.per_sm[dev];
        sms = setup.sms[dev];
    }
    dim3 block(TX * L::TYe);
    dim3 grid((C.n[0] + TX - 1) / TX, (DIM >= 2) ? (C.n[1] + TY - 1) / TY : 1, 1);
    int zchunk = 1;
    if (DIM == 3) {
        if (a.zchunk > 0) {
            zchunk = a.zchunk;
        } else {
            // split the z-march so that there are at least four CTAs per
            // resident slot; each chunk re-reads a 2-plane halo in z
            const long long tiles = (long long)grid.x * grid.y;
            const long long want = 4LL * per_sm * sms;
            const int chunks = (int)std::max(1LL, (want + tiles - 1) / tiles);
            zchunk = std::max(8, (C.n[2] + chunks - 1) / chunks);
        }
        grid.z = (C.n[2] + zchunk - 1) / zchunk;
    }
    kern<<<grid, block, L::BYTES, a.stream>>>(
        static_cast<const T*>(a.phi_in), static_cast<const T*>(a.c_in),
        static_cast<const T*>(a.d_in), static_cast<const T*>(a.clo_in), static_cast<const T*>(a.plo_in),
        static_cast<T*>(a.phi_out), static_cast<T*>(a.c_out), static_cast<T*>(a.d_out),
        static_cast<T*>(a.clo_out), static_cast<T*>(a.plo_out), C, K, zchunk);
    return cudaGetLastError();
}

template <typename T>
static Consts<T> make_consts(const HostProblem& P) {
    Consts<T> C;
    C.dim = P.dim;
    for (int a = 0; a < 3; ++a) {
        C.n[a] = (int)P.n[a];
        C.bc_lo[a] = P.bc_lo[a];
        C.bc_hi[a] = P.bc_hi[a];
    }
    C.interp = P.interp;
    C.lap = P.lap;
    C.mobility = P.mobility;
    C.dir_phi = T(P.dir_phi); C.dir_cs = T(P.dir_cs); C.dir_cl = T(P.dir_cl);
    C.dx = T(P.dx);
    C.inv_dx = T(1.0 / P.dx);
    C.inv_2dx = T(1.0 / (2.0 * P.dx));
    C.inv_dx2 = T(1.0 / (P.dx * P.dx));
    C.H = T(P.H); C.sigma = T(P.sigma); C.inv_Mphi = T(1.0 / P.M_phi);
    C.D_s = T(P.D_s); C.D_l = T(P.D_l);
    C.log_ke = T(std::log(P.k_e)); C.one_m_ke = T(1.0 - P.k_e);
    C.A = T(P.A); C.one_m_A = T(1.0 - P.A); C.b = T(P.b); C.a = T(P.a);
    C.delta2 = T(P.delta * P.delta);
    C.dt = T(P.dt);
    C.G_theta = T(P.G_theta);
    set_coefficients(C);
    return C;
}

template <typename T>
static Clock<T> make_clock(const HostProblem& P, int64_t step, int64_t shifts) {
    const double t = (double)step * P.dt;
    Clock<T> K;
    K.theta0 = T(P.theta_ref + P.G_theta * (P.x0 + P.v_pull * t - (double)shifts * P.dx));
    return K;
}

template <typename T>
static cudaError_t launch_T(const StepLaunch& a) {
    const HostProblem& P = *a.prob;
    const Consts<T> C = make_consts<T>(P);
    const Clock<T> K = make_clock<T>(P, a.step, a.shifts);
    // 1D: 32-cell tiles, so that a short line still spreads over many SMs
    // (a 1024-cell FP64 line is bound by the FP64 units of the SMs it runs on)
    if (P.dim == 1) return launch_tile<T, 1, 32, 1>(a, C, K);
    if (P.dim == 2) return a.use_generic ? launch_tile<T, 2, 32, 8>(a, C, K) : launch_step2d<T>(a, C, K);
    if (a.use_generic) return launch_tile<T, 3, 32, 8>(a, C, K);
    return launch_step3d<T>(a, C, K);
}

cudaError_t launch_step(const StepLaunch& a) {
    if (a.prob->precision == 1) return launch_T<double>(a);
    return launch_T<float>(a);
}

size_t step_smem_bytes(int precision, int dim) {
    if (precision == 1) {
        if (dim == 1) return Tile<double, 1, 32, 1>::BYTES;
        if (dim == 2) return Tile<double, 2, 32, 8>::BYTES;
        return Tile<double, 3, 32, 8>::BYTES;
    }
    if (dim == 1) return Tile<float, 1, 32, 1>::BYTES;
    if (dim == 2) return Tile<float, 2, 32, 8>::BYTES;
    return Tile<float, 3, 32, 8>::BYTES;
}

}  // namespace pf
