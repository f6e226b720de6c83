// pf_step3d.cu -- the fused explicit step for 3D grids (FP32 and FP64).
//
// Same method and discretisation as pf_step.cu (the brackets of Eqs.
// cs_nonvar / cl_nonvar at faces, Eq. phasefield_nonvar at cells with the
// re-derived driving force, conservative (c, d) update, forward Euler), laid
// out for throughput on one GB300:
//   * one CTA = a TX x TY tile of columns marching along z over a chunk of
//     planes; the grid has several chunks per column so that every SM holds
//     four CTAs;
//   * per z-plane, the halo-2 tile of each plane is loaded once and turned
//     into packed records {phi, Y, mu_s, mu_l} (16 B in FP32) and {c_s, c_l},
//     kept in shared-memory rings (4 planes of records, 3 of the rest; about
//     51 KB per CTA in FP32, so that four CTAs share an SM);
//   * centred gradients are not stored: a face builds its transverse
//     components from the packed records of its two cells' neighbours, so one
//     vector load serves all four fields;
//   * x, y and z faces of a plane are computed in one balanced loop, each face
//     once, and stored as (F_c, F_d) pairs;
//   * FP32 reciprocals use the hardware approximation (a few ulp), FP64 is
//     exact IEEE.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include "pf_internal.cuh"
#include "pf_kernels.h"

namespace pf {

template <typename T>
struct alignas(4 * sizeof(T)) V4 {
    T x, y, z, w;   // phi, Y, mu_s, mu_l
};
template <typename T>
struct alignas(2 * sizeof(T)) V2 {
    T x, y;
};

__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }

template <typename T, int TX, int TY>
struct Tile3 {
    static constexpr int NT = TX * TY;
    static constexpr int HX = TX + 4, HY = TY + 4, HP = HX * HY;   // halo-2 plane
    static constexpr int RX = TX + 2, RY = TY + 2, RP = RX * RY;   // ring-1 plane
    static constexpr int NS = 4;   // slots of packed records (planes z-1 .. z+2)
    static constexpr int N3 = 3;   // slots of {c_s, c_l} and phi (planes z .. z+2)
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1), NFZ = TX * TY;
    static constexpr int NF = NFX + NFY + NFZ;
    static constexpr size_t OFF_G4 = 0;
    static constexpr size_t OFF_C2 = OFF_G4 + sizeof(V4<T>) * NS * HP;
    static constexpr size_t OFF_PH = OFF_C2 + sizeof(V2<T>) * N3 * HP;
    static constexpr size_t OFF_PD = OFF_PH + sizeof(T) * N3 * HP;
    static constexpr size_t OFF_FX = OFF_PD + sizeof(T) * 2 * RP;
    static constexpr size_t OFF_FY = OFF_FX + sizeof(V2<T>) * NFX;
    static constexpr size_t OFF_FZ = OFF_FY + sizeof(V2<T>) * NFY;
    static constexpr size_t BYTES = OFF_FZ + sizeof(V2<T>) * NFZ;
};

// face fluxes from the face state; nrm = normal differences (R - L) of
// {phi, Y, mu_s, mu_l} times 1/dx, t1, t2 = the two transverse components.
// With T_i = M_i [d_a mu_i (|g_t|^2 + delta^2) - g_a (g_t . grad_t mu_i)] (the
// tangential fluxes times 1/r) and w_s + w_l = 1, p w_s - (1-p) w_l = a(phi):
//   F_c = r [q g_a (g . grad Y) + p T_s + (1-p) T_l + (1-A) d phidot g_a a(phi)]
//   F_d = r [T_s - T_l + (1-A) d phidot g_a]
template <typename T>
__device__ __forceinline__ V2<T> face3(const Consts<T>& C, T phiL, T phiR, V2<T> cL, V2<T> cR,
                                       T pdL, T pdR, V4<T> nrm, V4<T> t1, V4<T> t2) {
    const T f = T(0.5) * (phiL + phiR);
    const T cs = T(0.5) * (cL.x + cR.x);
    const T cl = T(0.5) * (cL.y + cR.y);
    const T d = cs - cl;
    const T pdot = T(0.5) * (pdL + pdR);
    const T p = p_of(C, f);
    const T omp = T(1) - p;
    const T Ms = Ms_of(C, cs), Ml = Ml_of(C, cl);
    const T bMl = C.b * Ml;
    const T iMbar = frcp(Ms * omp + bMl * p);
    const T gt2d = t1.x * t1.x + t2.x * t2.x + C.delta2;
    const T ga = nrm.x;
    const T r = frcp(ga * ga + gt2d);
    const T dY = ga * nrm.y + t1.x * t1.y + t2.x * t2.y;
    const T Ts = Ms * (nrm.z * gt2d - ga * (t1.x * t1.z + t2.x * t2.z));
    const T Tl = Ml * (nrm.w * gt2d - ga * (t1.x * t1.w + t2.x * t2.w));
    const T at = C.one_m_A * d * pdot * ga;
    const T q = Ms * Ml * (C.b * p + omp) * iMbar;
    const T afn = (Ms - bMl) * p * omp * iMbar;
    V2<T> out;
    out.x = r * (q * ga * dY + p * Ts + omp * Tl + at * afn);   // F_c
    out.y = r * (Ts - Tl + at);                                  // F_d
    return out;
}

template <typename T>
__device__ __forceinline__ V4<T> sub4(V4<T> a, V4<T> b) {
    return V4<T>{a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w};
}
template <typename T>
__device__ __forceinline__ V4<T> add4(V4<T> a, V4<T> b) {
    return V4<T>{a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w};
}
template <typename T>
__device__ __forceinline__ V4<T> scale4(V4<T> a, T s) {
    return V4<T>{a.x * s, a.y * s, a.z * s, a.w * s};
}

__device__ __forceinline__ int slot3(int z) { return ((z % 3) + 3) % 3; }

// Per-thread work lists, fixed for the whole z-march: each thread owns up to
// JH halo cells (plane loads), JR ring cells (phase-field rates) and JF faces.
template <int TX, int TY>
struct Work3 {
    static constexpr int NT = TX * TY;
    static constexpr int HX = TX + 4, HP = (TX + 4) * (TY + 4);
    static constexpr int RX = TX + 2, RP = (TX + 2) * (TY + 2);
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1), NFZ = TX * TY;
    static constexpr int NF = NFX + NFY + NFZ;
    static constexpr int JH = (HP + NT - 1) / NT;
    static constexpr int JR = (RP + NT - 1) / NT;
    static constexpr int JF = (NF + NT - 1) / NT;
};

// face descriptor packed in 32 bits: bits 0-11 left-cell halo index, 12-23
// left-cell ring index, 24-25 axis (0 x, 1 y, 2 z, 3 none), 26 no-flux face
__device__ __forceinline__ unsigned pack_face(int h, int r, int axis, bool nf) {
    return (unsigned)h | ((unsigned)r << 12) | ((unsigned)axis << 24) | ((unsigned)nf << 26);
}

template <typename T, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB)
step3d_kernel(const T* __restrict__ phi_in, const T* __restrict__ c_in,
              const T* __restrict__ d_in, const T* __restrict__ clo_in,
              T* __restrict__ phi_out, T* __restrict__ c_out, T* __restrict__ d_out,
              T* __restrict__ clo_out, Consts<T> C, Clock<T> K, int zchunk) {
    using L = Tile3<T, TX, TY>;
    using W = Work3<TX, TY>;
    static_assert(L::HP < 4096 && L::RP < 4096, "tile too large for the packed descriptors");
    extern __shared__ __align__(16) unsigned char smem[];
    V4<T>* sG4 = reinterpret_cast<V4<T>*>(smem + L::OFF_G4);
    V2<T>* sC2 = reinterpret_cast<V2<T>*>(smem + L::OFF_C2);
    T* sPh = reinterpret_cast<T*>(smem + L::OFF_PH);
    T* sPd = reinterpret_cast<T*>(smem + L::OFF_PD);
    V2<T>* sFx = reinterpret_cast<V2<T>*>(smem + L::OFF_FX);
    V2<T>* sFy = reinterpret_cast<V2<T>*>(smem + L::OFF_FY);
    V2<T>* sFz = reinterpret_cast<V2<T>*>(smem + L::OFF_FZ);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nx = C.n[0], ny = C.n[1], nz = C.n[2];
    const long long sz = (long long)nx * ny;
    const T q_inv_dx = T(0.25) * C.inv_dx;      // mean of two centred differences (f+ - f-)/(2 dx)

    // ---- work lists (independent of z)
    int hoff[W::JH];          // in-plane global offset of each owned halo cell, -1: Dirichlet ghost
#pragma unroll
    for (int j = 0; j < W::JH; ++j) {
        const int h = tid + j * W::NT;
        hoff[j] = -1;
        if (h < L::HP) {
            const int mx = map_coord(x0 - 2 + h % L::HX, nx, C.bc_lo[0], C.bc_hi[0]);
            const int my = map_coord(y0 - 2 + h / L::HX, ny, C.bc_lo[1], C.bc_hi[1]);
            if (mx >= 0 && my >= 0) hoff[j] = my * nx + mx;
        }
    }
    int rdesc[W::JR];         // halo index of each owned ring cell | Dirichlet flag << 12
    T rxc[W::JR];             // x coordinate of its (mapped) centre, for theta
#pragma unroll
    for (int j = 0; j < W::JR; ++j) {
        const int r = tid + j * W::NT;
        rdesc[j] = 0;
        rxc[j] = T(0);
        if (r < L::RP) {
            const int rx = r % L::RX, ry = r / L::RX;
            const int gx = x0 - 1 + rx;
            const int mx = map_coord(gx, nx, C.bc_lo[0], C.bc_hi[0]);
            const bool dir = mx < 0 || map_coord(y0 - 1 + ry, ny, C.bc_lo[1], C.bc_hi[1]) < 0;
            rdesc[j] = ((ry + 1) * L::HX + rx + 1) | ((int)dir << 12);
            rxc[j] = (T((mx < 0) ? gx : mx) + T(0.5)) * C.dx;
        }
    }
    unsigned fdesc[W::JF];
#pragma unroll
    for (int j = 0; j < W::JF; ++j) {
        const int f = tid + j * W::NT;
        fdesc[j] = pack_face(0, 0, 3, false);
        if (f < L::NFX) {
            const int fx = f % (TX + 1), fy = f / (TX + 1);
            const int gxl = x0 + fx - 1;
            const bool nf = (gxl == -1 && C.bc_lo[0] == BC_NOFLUX) || (gxl == nx - 1 && C.bc_hi[0] == BC_NOFLUX);
            fdesc[j] = pack_face((fy + 2) * L::HX + fx + 1, (fy + 1) * L::RX + fx, 0, nf);
        } else if (f < L::NFX + L::NFY) {
            const int e = f - L::NFX;
            const int fx = e % TX, fy = e / TX;
            const int gyl = y0 + fy - 1;
            const bool nf = (gyl == -1 && C.bc_lo[1] == BC_NOFLUX) || (gyl == ny - 1 && C.bc_hi[1] == BC_NOFLUX);
            fdesc[j] = pack_face((fy + 1) * L::HX + fx + 2, fy * L::RX + fx + 1, 1, nf);
        } else if (f < L::NF) {
            const int e = f - L::NFX - L::NFY;
            const int cx = e % TX, cy = e / TX;
            fdesc[j] = pack_face((cy + 2) * L::HX + cx + 2, (cy + 1) * L::RX + cx + 1, 2, false);
        }
    }
    const int own_h = (ty + 2) * L::HX + tx + 2;
    const int own_r = (ty + 1) * L::RX + tx + 1;
    const bool own_in = (x0 + tx < nx) && (y0 + ty < ny);
    const long long own_xy = (long long)(y0 + ty) * nx + (x0 + tx);

    // ---- A: plane z into the rings, from values fetched by fetch_plane
    T pf_f[W::JH], pf_c[W::JH], pf_d[W::JH];
    auto fetch_plane = [&](int z) {
        const int mz = map_coord(z, nz, C.bc_lo[2], C.bc_hi[2]);
#pragma unroll
        for (int j = 0; j < W::JH; ++j) {
            pf_f[j] = pf_c[j] = pf_d[j] = T(0);
            if (mz >= 0 && hoff[j] >= 0) {
                const long long gi = (long long)mz * sz + hoff[j];
                pf_f[j] = phi_in[gi];
                pf_c[j] = c_in[gi];
                pf_d[j] = d_in[gi];
            }
        }
    };
    auto store_plane = [&](int z) {
        const bool dirz = map_coord(z, nz, C.bc_lo[2], C.bc_hi[2]) < 0;
        V4<T>* g4 = sG4 + (z & 3) * L::HP;
        V2<T>* c2 = sC2 + slot3(z) * L::HP;
        T* ph = sPh + slot3(z) * L::HP;
#pragma unroll
        for (int j = 0; j < W::JH; ++j) {
            const int h = tid + j * W::NT;
            if (j * W::NT + W::NT > L::HP && h >= L::HP) break;
            T f, cs, cl, p;
            if (dirz || hoff[j] < 0) {
                f = C.dir_phi; cs = C.dir_cs; cl = C.dir_cl;
                p = p_of(C, f);
            } else {
                f = pf_f[j];
                p = p_of(C, f);
                cs = pf_c[j] + (T(1) - p) * pf_d[j];
                cl = pf_c[j] - p * pf_d[j];
            }
            const T mus = flog(cs) - C.log_ke;
            const T mul = flog(cl);
            g4[h] = V4<T>{f, mul + p * (mus - mul), mus, mul};
            c2[h] = V2<T>{cs, cl};
            ph[h] = f;
        }
    };

    // ---- B: phase-field rate of plane z on the ring-1 region -> sPd[z & 1]
    auto rates_plane = [&](int z) {
        const bool dirz = map_coord(z, nz, C.bc_lo[2], C.bc_hi[2]) < 0;
        T* pdz = sPd + (z & 1) * L::RP;
        const V4<T>* G0 = sG4 + (z & 3) * L::HP;
        const V4<T>* GM = sG4 + ((z - 1) & 3) * L::HP;
        const V4<T>* GP = sG4 + ((z + 1) & 3) * L::HP;
        const V2<T>* C0 = sC2 + slot3(z) * L::HP;
        const T* P0 = sPh + slot3(z) * L::HP;
        const T* PM = sPh + slot3(z - 1) * L::HP;
        const T* PP = sPh + slot3(z + 1) * L::HP;
#pragma unroll
        for (int j = 0; j < W::JR; ++j) {
            const int r = tid + j * W::NT;
            if (j * W::NT + W::NT > L::RP && r >= L::RP) break;
            const int h = rdesc[j] & 0xfff;
            T pd = T(0);
            if (!dirz && !(rdesc[j] >> 12)) {
                const V4<T> c0 = G0[h];
                const V4<T> ex = sub4(G0[h + 1], G0[h - 1]);
                const V4<T> ey = sub4(G0[h + L::HX], G0[h - L::HX]);
                const V4<T> ez = sub4(GP[h], GM[h]);
                const V2<T> cc = C0[h];
                const T fc = c0.x;
                const T faces = P0[h - 1] + P0[h + 1] + P0[h - L::HX] + P0[h + L::HX] + PM[h] + PP[h];
                T lap;
                if (C.lap == 7) {
                    lap = faces - T(6) * fc;
                } else {
                    const T edges = P0[h + L::HX + 1] + P0[h + L::HX - 1] + P0[h - L::HX + 1] +
                                    P0[h - L::HX - 1] + PP[h + 1] + PP[h - 1] + PM[h + 1] + PM[h - 1] +
                                    PP[h + L::HX] + PP[h - L::HX] + PM[h + L::HX] + PM[h - L::HX];
                    lap = T(1.0 / 3.0) * faces + T(1.0 / 6.0) * edges - T(4) * fc;
                }
                lap *= C.inv_dx2;
                const T cs = cc.x, cl = cc.y, mus = c0.z, mul = c0.w;
                const T p = p_of(C, fc), dp = dp_of(C, fc);
                const T Ms = Ms_of(C, cs), Ml = Ml_of(C, cl);
                const T bMl = C.b * Ml;
                const T Msq = Ms * (T(1) - p);
                const T iMbar = frcp(Msq + bMl * p);
                const T d = cs - cl;
                const T s2 = C.inv_2dx * C.inv_2dx;
                const T g2 = (ex.x * ex.x + ey.x * ey.x + ez.x * ez.x) * s2;
                const T cross = ((Ms * ex.z - bMl * ex.w) * ex.x + (Ms * ey.z - bMl * ey.w) * ey.x +
                                 (Ms * ez.z - bMl * ez.w) * ez.x) * s2;
                const T rr = frcp(g2 + C.delta2);
                const T pq = p * (T(1) - p);
                const T Kc = C.inv_Mphi + C.one_m_A * C.one_m_A * d * d * C.b * pq * rr * iMbar *
                                              frcp(C.b * p + T(1) - p);
                const T theta = K.theta0 - C.G_theta * rxc[j];
                const T dmu = mus - mul;
                // DeltaG = c_s (mu_s - mu_l) - d - (1-k_e) theta - D d (mu_s - mu_l)
                const T Dd = (Msq * (T(1) - C.A * (T(1) - p)) + C.A * bMl * p * p) * iMbar;
                const T dG = cs * dmu - d - C.one_m_ke * theta - Dd * d * dmu;
                const T dfdw = T(2) * fc * (T(1) - fc) * (T(1) - T(2) * fc);
                const T R = C.sigma * lap - C.H * dfdw - dG * dp + C.one_m_A * d * pq * iMbar * cross * rr;
                pd = R * frcp(Kc);
            }
            pdz[r] = pd;
        }
    };

    // ---- C: every face of plane z (x, y in the plane; z between z and z+1)
    auto faces_plane = [&](int z) {
        const V4<T>* G0 = sG4 + (z & 3) * L::HP;
        const V4<T>* GM = sG4 + ((z - 1) & 3) * L::HP;
        const V4<T>* GP = sG4 + ((z + 1) & 3) * L::HP;
        const V2<T>* C0 = sC2 + slot3(z) * L::HP;
        const V2<T>* CP = sC2 + slot3(z + 1) * L::HP;
        const T* pd0 = sPd + (z & 1) * L::RP;
        const T* pd1 = sPd + ((z + 1) & 1) * L::RP;
        const bool znf = (z == -1 && C.bc_lo[2] == BC_NOFLUX) || (z == nz - 1 && C.bc_hi[2] == BC_NOFLUX);
#pragma unroll
        for (int j = 0; j < W::JF; ++j) {
            const int f = tid + j * W::NT;
            const unsigned dsc = fdesc[j];
            const int axis = (dsc >> 24) & 3;
            if (axis == 3) break;
            const int hL = dsc & 0xfff, rL = (dsc >> 12) & 0xfff;
            const bool nf = (dsc >> 26) & 1;
            V2<T> F{T(0), T(0)};
            if (axis == 0) {
                if (!nf) {
                    const int hR = hL + 1;
                    const V4<T> aL = G0[hL], aR = G0[hR];
                    const V4<T> ty_ = scale4(add4(sub4(G0[hL + L::HX], G0[hL - L::HX]),
                                                  sub4(G0[hR + L::HX], G0[hR - L::HX])), q_inv_dx);
                    const V4<T> tz_ = scale4(add4(sub4(GP[hL], GM[hL]), sub4(GP[hR], GM[hR])), q_inv_dx);
                    F = face3(C, aL.x, aR.x, C0[hL], C0[hR], pd0[rL], pd0[rL + 1],
                              scale4(sub4(aR, aL), C.inv_dx), ty_, tz_);
                }
                sFx[f] = F;
            } else if (axis == 1) {
                if (!nf) {
                    const int hR = hL + L::HX;
                    const V4<T> aL = G0[hL], aR = G0[hR];
                    const V4<T> tx_ = scale4(add4(sub4(G0[hL + 1], G0[hL - 1]), sub4(G0[hR + 1], G0[hR - 1])),
                                             q_inv_dx);
                    const V4<T> tz_ = scale4(add4(sub4(GP[hL], GM[hL]), sub4(GP[hR], GM[hR])), q_inv_dx);
                    F = face3(C, aL.x, aR.x, C0[hL], C0[hR], pd0[rL], pd0[rL + L::RX],
                              scale4(sub4(aR, aL), C.inv_dx), tx_, tz_);
                }
                sFy[f - L::NFX] = F;
            } else {
                if (!znf) {
                    const V4<T> aL = G0[hL], aR = GP[hL];
                    const V4<T> tx_ = scale4(add4(sub4(G0[hL + 1], G0[hL - 1]), sub4(GP[hL + 1], GP[hL - 1])),
                                             q_inv_dx);
                    const V4<T> ty_ = scale4(add4(sub4(G0[hL + L::HX], G0[hL - L::HX]),
                                                  sub4(GP[hL + L::HX], GP[hL - L::HX])), q_inv_dx);
                    F = face3(C, aL.x, aR.x, C0[hL], CP[hL], pd0[rL], pd1[rL],
                              scale4(sub4(aR, aL), C.inv_dx), tx_, ty_);
                }
                sFz[f - L::NFX - L::NFY] = F;   // face (z, z+1)
            }
        }
    };

    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(nz, z0 + zchunk);
    if (z0 >= z1) return;

    // prologue: planes z0-2 .. z0+1, rates of z0-1 and z0, z faces (z0-1, z0);
    // plane z0+1 reuses the {c_s, c_l}/phi slot of z0-2, so it comes after rates(z0-1)
    for (int z = z0 - 2; z <= z0; ++z) {
        fetch_plane(z);
        store_plane(z);
    }
    fetch_plane(z0 + 1);
    __syncthreads();
    rates_plane(z0 - 1);
    __syncthreads();
    store_plane(z0 + 1);
    fetch_plane(z0 + 2);
    __syncthreads();
    rates_plane(z0);
    __syncthreads();
    faces_plane(z0 - 1);     // x/y faces of plane z0-1 are computed and unused
    __syncthreads();
    V2<T> fz_down = sFz[tid];

    // own-cell state of the plane being updated, fetched one iteration ahead
    T own_c = T(0), own_d = T(0), own_lo = T(0);
    auto fetch_own = [&](int z) {
        if (own_in && z < nz) {
            const long long gi = (long long)z * sz + own_xy;
            own_c = c_in[gi];
            own_d = d_in[gi];
            if (clo_in != nullptr) own_lo = clo_in[gi];
        }
    };
    fetch_own(z0);

    for (int k = z0; k < z1; ++k) {
        // plane k+2 arrived in registers during the previous iteration
        store_plane(k + 2);
        const T c_k = own_c, d_k = own_d, lo_k = own_lo;
        if (k + 1 < z1) {
            fetch_plane(k + 3);      // in flight during the rest of this iteration
            fetch_own(k + 1);
        }
        __syncthreads();
        rates_plane(k + 1);
        __syncthreads();
        faces_plane(k);
        __syncthreads();
        const V2<T> fz_up = sFz[tid];
        if (own_in) {
            const V2<T> fxl = sFx[ty * (TX + 1) + tx], fxr = sFx[ty * (TX + 1) + tx + 1];
            const V2<T> fyl = sFy[ty * TX + tx], fyr = sFy[(ty + 1) * TX + tx];
            const T dc = (fxr.x - fxl.x) + (fyr.x - fyl.x) + (fz_up.x - fz_down.x);
            const T dd = (fxr.y - fxl.y) + (fyr.y - fyl.y) + (fz_up.y - fz_down.y);
            const long long gi = (long long)k * sz + own_xy;
            const T dtdx = C.dt * C.inv_dx;
            const T dcv = dtdx * dc;
            phi_out[gi] = sG4[(k & 3) * L::HP + own_h].x + C.dt * sPd[(k & 1) * L::RP + own_r];
            d_out[gi] = d_k + dtdx * dd;
            if (clo_in != nullptr) {
                // compensated (TwoSum) update of c = hi + lo
                const T s = c_k + dcv;
                const T bv = s - c_k;
                const T err = (c_k - (s - bv)) + (dcv - bv);
                const T lo = lo_k + err;
                const T hi = s + lo;
                c_out[gi] = hi;
                clo_out[gi] = lo - (hi - s);
            } else {
                c_out[gi] = c_k + dcv;
            }
        }
        fz_down = fz_up;
    }
}

template <typename T, int TX, int TY, int MINB>
cudaError_t launch_step3d_tile(const StepLaunch& a, const Consts<T>& C, const Clock<T>& K) {
    using L = Tile3<T, TX, TY>;
    auto kern = step3d_kernel<T, TX, TY, MINB>;
    static bool configured = false;
    static int per_sm = 1, sms = 1;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, L::NT, L::BYTES);
        if (per_sm < 1) per_sm = 1;
        configured = true;
    }
    dim3 block(L::NT);
    dim3 grid((C.n[0] + TX - 1) / TX, (C.n[1] + TY - 1) / TY, 1);
    int zchunk = a.zchunk;
    if (zchunk <= 0) {
        const long long tiles = (long long)grid.x * grid.y;
        const long long want = 4LL * per_sm * sms;
        const int chunks = (int)std::max(1LL, (want + tiles - 1) / tiles);
        zchunk = std::max(8, (C.n[2] + chunks - 1) / chunks);
    }
    grid.z = (C.n[2] + zchunk - 1) / zchunk;
    kern<<<grid, block, L::BYTES, a.stream>>>(
        static_cast<const T*>(a.phi_in), static_cast<const T*>(a.c_in), static_cast<const T*>(a.d_in),
        static_cast<const T*>(a.clo_in), static_cast<T*>(a.phi_out), static_cast<T*>(a.c_out),
        static_cast<T*>(a.d_out), static_cast<T*>(a.clo_out), C, K, zchunk);
    return cudaGetLastError();
}

template cudaError_t launch_step3d_tile<float, 32, 8, 4>(const StepLaunch&, const Consts<float>&,
                                                         const Clock<float>&);
template cudaError_t launch_step3d_tile<double, 32, 8, 2>(const StepLaunch&, const Consts<double>&,
                                                          const Clock<double>&);

size_t step3d_smem_bytes(int precision) {
    return precision == 1 ? Tile3<double, 32, 8>::BYTES : Tile3<float, 32, 8>::BYTES;
}

}  // namespace pf
