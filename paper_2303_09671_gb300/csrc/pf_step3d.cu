// pf_step3d.cu -- the fused explicit step for 3D grids (FP32 and FP64).
//
// Same method and discretisation as pf_step.cu (the brackets of Eqs.
// cs_nonvar / cl_nonvar at faces, Eq. phasefield_nonvar at cells with the
// re-derived driving force, conservative (c, d) update, forward Euler), laid
// out for throughput on one GB300:
//   * a CTA owns a TX x TY tile of columns (TY even) and marches along z over a
//     chunk of planes; thread (tx, ty) owns the two cells (x, y) and (x, y+1),
//     y = y0 + 2 ty, and evaluates everything for both at once as a two-lane
//     vector.  In FP32 the lanes are the packed .f32x2 add/mul/fma of sm_100
//     class GPUs, which do two FP32 operations per issue slot;
//   * shared memory holds the halo-2 tile of each plane as two-lane records
//     {phi, Y}, {mu_s, mu_l}, {c_s, c_l} and phi (rings of 4, 4, 3 and 3
//     planes), the phase-field rate on the halo-1 ring (2 planes) and the
//     fluxes through the x faces and the upper y face of every cell pair; the
//     next plane arrives in a staging slot, in FP32 as tensor-memory-
//     accelerator boxes (cp.async.bulk.tensor on an mbarrier, issued by one
//     thread; waits bounded in time), else by per-cell cp.async copies; in
//     FP32 the updated plane leaves as TMA box stores from a shared tile;
//   * every thread evaluates the x+1/2, y+1/2 and z+1/2 faces of its own two
//     cells, so the neighbour records the three faces share are read once;
//     the faces on the tile's low x and low y edges are evaluated by warps 0
//     and 4;
//   * a y shift by one cell moves data between the lanes of neighbouring
//     records; those values are assembled lane by lane, everything else is
//     two-lane arithmetic;
//   * differences are kept in grid units (not divided by dx) and the stored
//     rate is dx^2 dphi/dt, so that F_c, F_d below are dx times the fluxes of
//     the model and the update is c += dt/dx^2 sum(F+ - F-);
//   * FP32 reciprocals and logarithms use the hardware approximations (a few
//     ulp), FP64 is exact IEEE.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include "pf_internal.cuh"
#include "pf_kernels.h"
#include "pf_lanes.cuh"
#include "pf_tma.cuh"

namespace pf {

template <typename T, int TX, int TY>
struct PTile {
    static_assert(TY % 2 == 0, "cells are paired along y");
    using V = typename Lanes<T>::V;
    using Q = Q2<V>;
    static constexpr int TYP = TY / 2;                  // pair rows
    static constexpr int NT = TX * TYP;                 // threads
    static constexpr int HW = TX + 4, HYP = TYP + 2;    // halo-2 plane: HW x HYP pair cells
    static constexpr int NH = HW * HYP;
    static constexpr int RW = TX + 2, NR = RW * HYP;    // halo-1 ring (all pair rows)
    // Row pitch of the plane arrays (measured: an odd pitch TX + 5 and a
    // 128-byte-aligned pitch TX + 8 were both slower than the dense TX + 4,
    // the latter also with the threads' own records 128-byte aligned: 8.6 %).
    static constexpr int HX = HW, RX = HX;
    static constexpr int OQ = 0, OV = 0, OD = 0, OF = 0;    // base shifts (elements)
    static constexpr int HP = HX * HYP, RP = HP;            // plane stride
    static constexpr int FXP = TX + 1;                      // x-face row pitch
    static constexpr int JH = (NH + NT - 1) / NT;
    static constexpr size_t OFF_A = 0;                                   // {phi, Y}, 4 planes
    static constexpr size_t OFF_B = OFF_A + sizeof(Q) * 4 * HP;          // {mu_s, mu_l}, 4 planes
    static constexpr size_t OFF_C = OFF_B + sizeof(Q) * 4 * HP;          // {c_s, c_l}, 3 planes
    static constexpr size_t OFF_P = OFF_C + sizeof(Q) * 3 * HP;          // phi, 3 planes
    static constexpr size_t OFF_D = OFF_P + sizeof(V) * 3 * HP;          // dx^2 phidot, 2 planes
    static constexpr size_t OFF_FX = OFF_D + sizeof(V) * 2 * RP;         // x faces {F_c, F_d}
    static constexpr size_t OFF_FY = OFF_FX + sizeof(Q) * (TYP * FXP);       // upper y face {F_c, F_d}
    // Staging of one plane.  TMA: the box of cells x0-4 .. x0+TX+3, y0-2 ..
    // y0+TY+1 per field, as the tensor-memory accelerator writes it (rows of
    // BXW elements; x starts 4 cells left of the tile so that the box's first
    // element is 16-byte aligned), each field's box followed by a slot for the
    // Dirichlet state (field stride RS, 128-byte aligned); the own state of the
    // plane being updated in boxes of the same shape.  cp.async: the pair
    // cells lane-planar, [field][lane][NHP], and the own state [field][lane][NT].
    static constexpr int BXW = TX + 8, BH = TY + 4, BOX = BXW * BH;
    static constexpr int RS = BOX + 128 / (int)sizeof(T);
    static constexpr int NHP = (NH + 15) / 16 * 16;
    static constexpr size_t OFF_R = (OFF_FY + sizeof(V) * (TYP + 1) * TX + 127) / 128 * 128;   // phi, c, d
    static constexpr size_t OFF_O = OFF_R + sizeof(T) * 3 * RS;                               // c, d, c_lo
    static constexpr size_t OFF_BAR = OFF_O + sizeof(T) * 3 * RS;                             // mbarrier
    // the updated plane of the tile (phi, c, d, c_lo: TX x TY each), written
    // back by TMA box stores
    static constexpr size_t OFF_W = (OFF_BAR + 16 + 127) / 128 * 128;
    static constexpr size_t BYTES = OFF_W + sizeof(T) * 4 * TX * TY;
    static_assert((sizeof(T) * RS) % 128 == 0 && OFF_BAR % 8 == 0, "staging boxes 128-byte aligned");
    // the per-cell layout needs less: the rest of the SM's 228 KB stays L1,
    // which its cp.async copies pass through
    static constexpr size_t OFF_R_CP = OFF_FY + sizeof(V) * (TYP + 1) * TX;
    static constexpr size_t OFF_O_CP = OFF_R_CP + sizeof(T) * 6 * NHP;
    static constexpr size_t BYTES_CP = OFF_O_CP + sizeof(T) * 6 * NT;
    static constexpr int NB = NR - NT;   // ring cells besides the threads' own pairs
    static_assert(NB == 2 * RW + 2 * TYP && NB <= NT, "ring = own pairs + border");
};

__device__ __forceinline__ int slot3(int z) { return ((z % 3) + 3) % 3; }

template <typename T, int TX, int TY, bool L19, bool AI, bool STD, bool TMA>
__global__ void __launch_bounds__(TX * (TY / 2), (sizeof(T) == 4 ? 2 : 1))
step3d_kernel(const T* __restrict__ phi_in, const T* __restrict__ c_in, const T* __restrict__ d_in,
              const T* __restrict__ clo_in, T* __restrict__ phi_out, T* __restrict__ c_out,
              T* __restrict__ d_out, T* __restrict__ clo_out, const PairConsts<typename Lanes<T>::V> K,
              const GridConsts<T> G, int zchunk, int zbase, const __grid_constant__ CUtensorMap tm_phi,
              const __grid_constant__ CUtensorMap tm_c, const __grid_constant__ CUtensorMap tm_d,
              const __grid_constant__ CUtensorMap tm_clo, const __grid_constant__ CUtensorMap tw_phi,
              const __grid_constant__ CUtensorMap tw_c, const __grid_constant__ CUtensorMap tw_d,
              const __grid_constant__ CUtensorMap tw_clo, int flags, int zpad, int* __restrict__ err) {
    using L = PTile<T, TX, TY>;
    using V = typename L::V;
    using Q = typename L::Q;
    constexpr int HX = L::HX, HP = L::HP, RX = L::RX, RP = L::RP, NT = L::NT, TYP = L::TYP;
    constexpr int HW = L::HW, NH = L::NH, NHP = L::NHP, RW = L::RW, FXP = L::FXP;
    constexpr int BXW = L::BXW, BH = L::BH, BOX = L::BOX, RS = L::RS;
    static_assert(HP < 4096, "tile too large for the packed ring descriptors");
    static_assert(NT >= 128 + TX && TYP <= 32, "edge faces need warps 0 and 4");
    extern __shared__ __align__(128) unsigned char smem[];
    Q* sA = reinterpret_cast<Q*>(smem + L::OFF_A) + L::OQ;
    Q* sB = reinterpret_cast<Q*>(smem + L::OFF_B) + L::OQ;
    Q* sC = reinterpret_cast<Q*>(smem + L::OFF_C) + L::OQ;
    V* sP = reinterpret_cast<V*>(smem + L::OFF_P) + L::OV;
    V* sD = reinterpret_cast<V*>(smem + L::OFF_D) + L::OD;
    Q* sFx = reinterpret_cast<Q*>(smem + L::OFF_FX) + L::OF;
    V* sFy = reinterpret_cast<V*>(smem + L::OFF_FY);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const long long sz = (long long)nx * ny;

    // ---- work lists, fixed for the whole z-march
    // halo pair cells this thread converts (pair index tid + j NT, ring index
    // hring[j] in the pitched plane arrays).  TMA: the plane arrives as a box
    // per field (one thread issues it) and loc[j][l] is the box index of the
    // source of row l of each pair cell (a mirror ghost's image lies inside the
    // box; cells further than the ghost width from the domain, present in
    // partial tiles only and never used by a cell of the domain, read any cell
    // of the box that lies in the domain), RS - 1 for a Dirichlet ghost (the
    // slot after each field's box holds the Dirichlet state).  Otherwise each
    // thread copies its cells with cp.async and loc[j][l] is the in-plane
    // offset of the source, -1 for a Dirichlet ghost.
    int loc[L::JH][2];
    int hring[L::JH];
#pragma unroll
    for (int j = 0; j < L::JH; ++j) {
        const int h = tid + j * NT;
        loc[j][0] = loc[j][1] = TMA ? RS - 1 : -1;
        hring[j] = (h / HW) * HX + h % HW;
        if (h < NH) {
            const int mx = map_coord(x0 - 2 + h % HW, nx, G.bc_lo[0], G.bc_hi[0]);
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const int my = map_coord(y0 - 2 + 2 * (h / HW) + l, ny, G.bc_lo[1], G.bc_hi[1]);
                if (mx < 0 || my < 0) continue;
                if constexpr (TMA) {
                    const int bx = min(max(mx - (x0 - 4), 0), BXW - 1);
                    const int by = min(max(my - (y0 - 2), 0), BH - 1);
                    loc[j][l] = by * BXW + bx;
                } else {
                    loc[j][l] = my * nx + mx;
                }
            }
        }
    }
    // ring cells: every thread its own pair, the last NB threads one border cell.
    // descriptor = halo index | ghost lanes << 12, 13 | first, last pair row << 14, 15
    auto ring_desc = [&](int rx, int ry, int& dsc, T& xc) {
        const int gx = x0 - 1 + rx;
        const int mx = map_coord(gx, nx, G.bc_lo[0], G.bc_hi[0]);
        const bool glo = mx < 0 || map_coord(y0 - 2 + 2 * ry, ny, G.bc_lo[1], G.bc_hi[1]) < 0;
        const bool ghi = mx < 0 || map_coord(y0 - 1 + 2 * ry, ny, G.bc_lo[1], G.bc_hi[1]) < 0;
        dsc = (ry * HX + rx + 1) | ((int)glo << 12) | ((int)ghi << 13) | ((int)(ry == 0) << 14) |
              ((int)(ry == L::HYP - 1) << 15);
        xc = (T((mx < 0) ? gx : mx) + T(0.5)) * G.dx;   // theta at the mirror / wrap image
    };
    int own_dsc, bor_dsc = 0, bor_r = -1;
    T own_xc, bor_xc = T(0);
    ring_desc(tx + 1, ty + 1, own_dsc, own_xc);
    constexpr int NB = L::NB;
    if (tid >= NT - NB) {
        const int b = tid - (NT - NB);
        int rx, ry;
        if (b < RW) { rx = b; ry = 0; }
        else if (b < 2 * RW) { rx = b - RW; ry = L::HYP - 1; }
        else if (b < 2 * RW + TYP) { rx = 0; ry = 1 + b - 2 * RW; }
        else { rx = RW - 1; ry = 1 + b - 2 * RW - TYP; }
        ring_desc(rx, ry, bor_dsc, bor_xc);
        bor_r = ry * RX + rx;
    }
    const int own_h = (ty + 1) * HX + tx + 2;
    const int own_r = (ty + 1) * RX + tx + 1;
    const int own_x = x0 + tx, own_y = y0 + 2 * ty;
    const bool in_lo = own_x < nx && own_y < ny;
    const bool in_hi = own_x < nx && own_y + 1 < ny;
    const long long own_xy = (long long)own_y * nx + own_x;
    const bool nf_x = own_x == nx - 1 && G.bc_hi[0] == BC_NOFLUX;
    const bool nf_ylo = own_y == ny - 1 && G.bc_hi[1] == BC_NOFLUX;
    const bool nf_yhi = own_y + 1 == ny - 1 && G.bc_hi[1] == BC_NOFLUX;
    const bool nf_x_edge = x0 == 0 && G.bc_lo[0] == BC_NOFLUX;
    const bool nf_y_edge = y0 == 0 && G.bc_lo[1] == BC_NOFLUX;

    // ---- A: plane z -> staging.
    // TMA: thread 0 issues the box of each field and the own-state boxes on one
    // mbarrier; every thread waits for its phase (bounded).  A Dirichlet ghost
    // plane is not copied: every thread writes the Dirichlet state where its
    // cells read.  Staging [field][RS]: the box (rows of BXW), then the slot
    // holding the Dirichlet state.
    // cp.async: each thread copies the cells it converts, lane-planar
    // ([field][lane][h]: consecutive threads write consecutive words), the own
    // state [field][lane][tid]; Dirichlet ghosts are written directly.
    T* sR = reinterpret_cast<T*>(smem + (TMA ? L::OFF_R : L::OFF_R_CP));
    T* sO = reinterpret_cast<T*>(smem + (TMA ? L::OFF_O : L::OFF_O_CP));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
    T* sW = reinterpret_cast<T*>(smem + L::OFF_W);   // [field][TY][TX]: the updated plane
    unsigned phase = 0;        // parity of the mbarrier phase waited for next
    bool timed_out = false;    // a wait ran out: no further arrivals, copies or waits
    unsigned stuck = 0;        // the parity of the phase that did not complete
    if constexpr (TMA) {
        if (tid == 0) mbar_init(bar, 1);
        if (tid < 3) sR[tid * RS + RS - 1] = tid == 0 ? G.dir_phi : (tid == 1 ? G.dir_c : G.dir_d);
        __syncthreads();
    }
    constexpr unsigned HALO_TX = 3u * BOX * sizeof(T);
    constexpr unsigned OWN_TX = (sizeof(T) == 4 ? 3u : 2u) * BOX * sizeof(T);
    // plane z into the staging slot (if plane), own state of plane zown (if >= 0)
    auto fetch = [&](int z, bool plane, int zown) {
        const int mz = plane ? map_coord(z, nz, G.bc_lo[2], G.bc_hi[2]) : 0;
        const bool copy_plane = plane && mz != DIR_GHOST;
        if constexpr (TMA) {
            if (plane && !copy_plane) {
#pragma unroll
                for (int j = 0; j < L::JH; ++j) {
                    if ((j + 1) * NT > NH && tid + j * NT >= NH) break;
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        sR[loc[j][l]] = G.dir_phi;
                        sR[RS + loc[j][l]] = G.dir_c;
                        sR[2 * RS + loc[j][l]] = G.dir_d;
                    }
                }
                fence_proxy_async_smem();   // before later TMA writes to the same slots
            }
            if (tid == 0 && !timed_out) {
                fence_proxy_async_smem();
                mbar_arrive_expect(bar, (copy_plane ? HALO_TX : 0u) + (zown >= 0 ? OWN_TX : 0u));
                if (!(flags & 2)) {   // flags bit 1: copies left out (a test of the bounded wait)
                    if (copy_plane) {
                        tma_load_3d(sR, &tm_phi, x0 - 4, y0 - 2, mz + zpad, bar);
                        tma_load_3d(sR + RS, &tm_c, x0 - 4, y0 - 2, mz + zpad, bar);
                        tma_load_3d(sR + 2 * RS, &tm_d, x0 - 4, y0 - 2, mz + zpad, bar);
                    }
                    if (zown >= 0) {
                        tma_load_3d(sO, &tm_c, x0 - 4, y0 - 2, zown + zpad, bar);
                        tma_load_3d(sO + RS, &tm_d, x0 - 4, y0 - 2, zown + zpad, bar);
                        if constexpr (sizeof(T) == 4)
                            tma_load_3d(sO + 2 * RS, &tm_clo, x0 - 4, y0 - 2, zown + zpad, bar);
                    }
                }
            }
        } else {
            if (plane) {
#pragma unroll
                for (int j = 0; j < L::JH; ++j) {
                    const int h = tid + j * NT;
                    if ((j + 1) * NT > NH && h >= NH) break;
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        T* dst = sR + l * NHP + h;
                        if (copy_plane && loc[j][l] >= 0) {
                            const long long gi = (long long)mz * sz + loc[j][l];
                            cp_async(dst, phi_in + gi);
                            cp_async(dst + 2 * NHP, c_in + gi);
                            cp_async(dst + 4 * NHP, d_in + gi);
                        } else {
                            dst[0] = G.dir_phi;
                            dst[2 * NHP] = G.dir_c;
                            dst[4 * NHP] = G.dir_d;
                        }
                    }
                }
            }
            if (zown >= 0) {
                const long long gi = (long long)zown * sz + own_xy;
                T* dst = sO + tid;
                if (in_lo) {
                    cp_async(dst, c_in + gi);
                    cp_async(dst + 2 * NT, d_in + gi);
                    if constexpr (sizeof(T) == 4) cp_async(dst + 4 * NT, clo_in + gi);
                }
                if (in_hi) {
                    cp_async(dst + NT, c_in + gi + nx);
                    cp_async(dst + 3 * NT, d_in + gi + nx);
                    if constexpr (sizeof(T) == 4) cp_async(dst + 5 * NT, clo_in + gi + nx);
                }
            }
            cp_async_commit();
        }
    };
    // wait for the last fetch
    auto fetched = [&]() {
        if constexpr (TMA) {
            if (!timed_out && !mbar_wait_bounded(bar, phase)) {
                timed_out = true;
                stuck = phase;
                if (err) atomicOr(err, 1);
            }
            phase ^= 1u;
        } else {
            cp_async_wait_all();
        }
    };
    // own state of the plane being updated: rows y and y+1 of the thread's pair
    auto own_state = [&](int f, int l) -> T {
        if constexpr (TMA) return sO[f * RS + (2 * ty + l + 2) * BXW + tx + 4];
        else return sO[(2 * f + l) * NT + tid];
    };
    // staged plane z into the rings
    auto store_plane = [&](int oa, int oc) {
        Q* A = sA + oa;
        Q* B = sB + oa;
        Q* C = sC + oc;
        V* P = sP + oc;
#pragma unroll
        for (int j = 0; j < L::JH; ++j) {
            const int hl = tid + j * NT;
            if ((j + 1) * NT > NH && hl >= NH) break;
            V f, c, d;
            if constexpr (TMA) {
                f = vpair(sR[loc[j][0]], sR[loc[j][1]]);
                c = vpair(sR[RS + loc[j][0]], sR[RS + loc[j][1]]);
                d = vpair(sR[2 * RS + loc[j][0]], sR[2 * RS + loc[j][1]]);
            } else {
                f = vpair(sR[hl], sR[NHP + hl]);
                c = vpair(sR[2 * NHP + hl], sR[3 * NHP + hl]);
                d = vpair(sR[4 * NHP + hl], sR[5 * NHP + hl]);
            }
            const int h = hring[j];
            const V p = vp_of<AI, STD>(K, f);
            const V cs = vfma(vsub(vlit<V>(1.0), p), d, c);
            const V cl = vsub(c, vmul(p, d));
            const V mus = vsub(vlog(cs), K.log_ke);
            const V mul = vlog(cl);
            A[h] = Q{f, vfma(p, vsub(mus, mul), mul)};
            B[h] = Q{mus, mul};
            C[h] = Q{cs, cl};
            P[h] = f;
        }
    };

    // ---- B: dx^2 phidot of one ring pair cell of plane z -> sD[z & 1][r]
    // rate of plane z: ring offsets of planes z-1, z, z+1 (A/B rings: am, a0, ap;
    // C/P rings: cm, c0, cp)
    auto rate_of = [&](bool ghost_z, int am, int a0, int ap, int cm, int c0, int cp, int dsc, T xc) -> V {
        const V* P0 = sP + c0;
        const V* PM = sP + cm;
        const V* PP = sP + cp;
        const Q* B0 = sB + a0;
        const Q* BM = sB + am;
        const Q* BP = sB + ap;
        const Q* C0 = sC + c0;
        const int h = dsc & 0xfff;
        const int hS = ((dsc >> 14) & 1) ? h : h - HX;   // first pair row: row below unused
        const int hN = ((dsc >> 15) & 1) ? h : h + HX;   // last pair row: row above unused
        V pd = vpair(T(0), T(0));
        if (!ghost_z) {
            const V f = P0[h];
            const V fxm = P0[h - 1], fxp = P0[h + 1], fS = P0[hS], fN = P0[hN];
            const V fzm = PM[h], fzp = PP[h];
            const V XP = vadd(fxm, fxp), ZP = vadd(fzm, fzp);
            const V YF = vpair(fS.y + f.y, f.x + fN.x);
            V lap;
            if (L19) {
                const V XS = vadd(P0[hS - 1], P0[hS + 1]), XN = vadd(P0[hN - 1], P0[hN + 1]);
                const V ZS = vadd(PM[hS], PP[hS]), ZN = vadd(PM[hN], PP[hN]);
                const V EXY = vpair(XS.y + XP.y, XP.x + XN.x);
                const V EZY = vpair(ZS.y + ZP.y, ZP.x + ZN.x);
                const V EXZ = vadd(vadd(PM[h - 1], PM[h + 1]), vadd(PP[h - 1], PP[h + 1]));
                lap = vsub(vfma(vlit<V>((1.0 / 3)), vadd(vadd(XP, ZP), YF), vmul(vlit<V>((1.0 / 6)), vadd(vadd(EXY, EZY), EXZ))),
                           vmul(vlit<V>(4.0), f));
            } else {
                lap = vsub(vadd(vadd(XP, ZP), YF), vmul(vlit<V>(6.0), f));
            }
            const Q cc = C0[h], bc = B0[h];
            const Q bxm = B0[h - 1], bxp = B0[h + 1], bS = B0[hS], bN = B0[hN], bzm = BM[h], bzp = BP[h];
            // centred differences (times 2 dx) of phi, mu_s, mu_l
            const V gx = vsub(fxp, fxm), gy = vpair(f.y - fS.y, fN.x - f.x), gz = vsub(fzp, fzm);
            const V sx = vsub(bxp.a, bxm.a), sy = vpair(bc.a.y - bS.a.y, bN.a.x - bc.a.x), sz_ = vsub(bzp.a, bzm.a);
            const V lx = vsub(bxp.b, bxm.b), ly = vpair(bc.b.y - bS.b.y, bN.b.x - bc.b.x), lz = vsub(bzp.b, bzm.b);
            const V cs = cc.a, cl = cc.b, mus = bc.a, mul = bc.b;
            const V p = vp_of<AI, STD>(K, f), dp = vdp_of<AI, STD>(K, f);
            const V omp = vsub(vlit<V>(1.0), p);
            const V Ms = STD ? vmul(K.Ms_c, cs) : vfma(K.Ms_c, cs, K.Ms_0);
            const V Ml = STD ? vmul(K.Ml_c, cl) : vfma(K.Ml_c, cl, K.Ml_0);
            const V bMl = vmul(K.b, Ml);
            const V Msq = vmul(Ms, omp);
            const V iMbar = vrcp(vfma(bMl, p, Msq));
            const V d = vsub(cs, cl);
            const V g2 = vfma(gx, gx, vfma(gy, gy, vmul(gz, gz)));
            const V ds = vfma(sx, gx, vfma(sy, gy, vmul(sz_, gz)));
            const V dl = vfma(lx, gx, vfma(ly, gy, vmul(lz, gz)));
            const V cross = vsub(vmul(Ms, ds), vmul(bMl, dl));     // (M_s grad mu_s - b M_l grad mu_l).grad phi
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
            pd = vmask(vmul(R, vrcp(Kc)), (dsc >> 12) & 1, (dsc >> 13) & 1);
        }
        return pd;
    };
    auto offA = [&](int z) { return (z & 3) * HP; };
    auto offC = [&](int z) { return slot3(z) * HP; };
    auto offD = [&](int z) { return (z & 1) * RP; };
    auto ghost = [&](int z) { return map_coord(z, nz, G.bc_lo[2], G.bc_hi[2]) == DIR_GHOST; };
    auto rate_z = [&](int z, int dsc, T xc) -> V {
        return rate_of(ghost(z), offA(z - 1), offA(z), offA(z + 1), offC(z - 1), offC(z), offC(z + 1), dsc, xc);
    };
    auto rate_cell = [&](int z, int dsc, T xc, int r) { sD[offD(z) + r] = rate_z(z, dsc, xc); };
    auto rates_plane = [&](int z) {
        rate_cell(z, own_dsc, own_xc, own_r);
        if (bor_r >= 0) rate_cell(z, bor_dsc, bor_xc, bor_r);
    };

    // ---- C: faces.  Components 0..3 = phi, Y, mu_s, mu_l = (A.a, A.b, B.a, B.b).
    // The cores take the records they read as arguments: the thread's own three
    // faces share most of them, and each is then read from shared memory once.
    // x face between halo cells L and R = L + 1: n = R - L; t1 (y) and t2 (z) =
    // the sums of the two cells' centred differences, from the rows S, N and the
    // planes M, P of both cells
    auto xface_core = [&](const Q& aL, const Q& bL, const Q& aR, const Q& bR, const Q& aS, const Q& bS,
                          const Q& aS1, const Q& bS1, const Q& aN, const Q& bN, const Q& aN1, const Q& bN1,
                          const Q& aPL, const Q& bPL, const Q& aPR, const Q& bPR, const Q& aML, const Q& bML,
                          const Q& aMR, const Q& bMR, const Q& cL, const Q& cR, const V dL, const V dR, V& Fc,
                          V& Fd) {
        V n[4] = {vsub(aR.a, aL.a), vsub(aR.b, aL.b), vsub(bR.a, bL.a), vsub(bR.b, bL.b)};
        // y: the rows of a pair are its two lanes
        V SP[4] = {vadd(aL.a, aR.a), vadd(aL.b, aR.b), vadd(bL.a, bR.a), vadd(bL.b, bR.b)};
        V SS[4] = {vadd(aS.a, aS1.a), vadd(aS.b, aS1.b), vadd(bS.a, bS1.a), vadd(bS.b, bS1.b)};
        V SN[4] = {vadd(aN.a, aN1.a), vadd(aN.b, aN1.b), vadd(bN.a, bN1.a), vadd(bN.b, bN1.b)};
        V t1[4], t2[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) t1[k] = vpair(SP[k].y - SS[k].y, SN[k].x - SP[k].x);
        t2[0] = vsub(vadd(aPL.a, aPR.a), vadd(aML.a, aMR.a));
        t2[1] = vsub(vadd(aPL.b, aPR.b), vadd(aML.b, aMR.b));
        t2[2] = vsub(vadd(bPL.a, bPR.a), vadd(bML.a, bMR.a));
        t2[3] = vsub(vadd(bPL.b, bPR.b), vadd(bML.b, bMR.b));
        face_flux<V, true, AI, STD>(K, vmul(vlit<V>(0.5), SP[0]), vadd(cL.a, cR.a), vadd(cL.b, cR.b), vadd(dL, dR), n,
                               t1, t2, Fc, Fd);
    };
    // y faces above the two rows of the pair P (lanes: y+1/2 inside P, y+3/2
    // between P and the pair N above): x differences from the E and W
    // neighbours of P and N, z differences from the planes U (z+1) and D (z-1)
    auto yface_core = [&](const Q& aP, const Q& bP, const Q& aN, const Q& bN, const Q& aPp, const Q& bPp,
                          const Q& aPm, const Q& bPm, const Q& aNp, const Q& bNp, const Q& aNm, const Q& bNm,
                          const Q& aPu, const Q& bPu, const Q& aPd, const Q& bPd, const Q& aNu, const Q& bNu,
                          const Q& aNd, const Q& bNd, const Q& cP_, const Q& cN_, const V dP, const V dN, V& Fc,
                          V& Fd) {
        const V cP[4] = {aP.a, aP.b, bP.a, bP.b};
        const V cN[4] = {aN.a, aN.b, bN.a, bN.b};
        V n[4], t1[4], t2[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) n[k] = vpair(cP[k].y - cP[k].x, cN[k].x - cP[k].y);
        const V DP[4] = {vsub(aPp.a, aPm.a), vsub(aPp.b, aPm.b), vsub(bPp.a, bPm.a), vsub(bPp.b, bPm.b)};
        const V DN[4] = {vsub(aNp.a, aNm.a), vsub(aNp.b, aNm.b), vsub(bNp.a, bNm.a), vsub(bNp.b, bNm.b)};
#pragma unroll
        for (int k = 0; k < 4; ++k) t1[k] = vpair(DP[k].x + DP[k].y, DP[k].y + DN[k].x);
        const V EP[4] = {vsub(aPu.a, aPd.a), vsub(aPu.b, aPd.b), vsub(bPu.a, bPd.a), vsub(bPu.b, bPd.b)};
        const V EN[4] = {vsub(aNu.a, aNd.a), vsub(aNu.b, aNd.b), vsub(bNu.a, bNd.a), vsub(bNu.b, bNd.b)};
#pragma unroll
        for (int k = 0; k < 4; ++k) t2[k] = vpair(EP[k].x + EP[k].y, EP[k].y + EN[k].x);
        const V f = vmul(vlit<V>(0.5), vpair(cP[0].x + cP[0].y, cP[0].y + cN[0].x));
        const V cs2 = vpair(cP_.a.x + cP_.a.y, cP_.a.y + cN_.a.x);
        const V cl2 = vpair(cP_.b.x + cP_.b.y, cP_.b.y + cN_.b.x);
        face_flux<V, true, AI, STD>(K, f, cs2, cl2, vpair(dP.x + dP.y, dP.y + dN.x), n, t1, t2, Fc, Fd);
    };
    // z face between the cell 0 on plane z and the cell 1 on plane z+1: x and y
    // differences from the E/W (p/m) and N/S neighbours on both planes
    auto zface_core = [&](const Q& a0, const Q& b0, const Q& a1, const Q& b1, const Q& ap0, const Q& bp0,
                          const Q& am0, const Q& bm0, const Q& ap1, const Q& bp1, const Q& am1, const Q& bm1,
                          const Q& aS0, const Q& bS0, const Q& aS1, const Q& bS1, const Q& aN0, const Q& bN0,
                          const Q& aN1, const Q& bN1, const Q& c0, const Q& c1, const V d0, const V d1, V& Fc,
                          V& Fd) {
        V n[4] = {vsub(a1.a, a0.a), vsub(a1.b, a0.b), vsub(b1.a, b0.a), vsub(b1.b, b0.b)};
        V t1[4], t2[4];
        t1[0] = vsub(vadd(ap0.a, ap1.a), vadd(am0.a, am1.a));
        t1[1] = vsub(vadd(ap0.b, ap1.b), vadd(am0.b, am1.b));
        t1[2] = vsub(vadd(bp0.a, bp1.a), vadd(bm0.a, bm1.a));
        t1[3] = vsub(vadd(bp0.b, bp1.b), vadd(bm0.b, bm1.b));
        const V SP[4] = {vadd(a0.a, a1.a), vadd(a0.b, a1.b), vadd(b0.a, b1.a), vadd(b0.b, b1.b)};
        const V SS[4] = {vadd(aS0.a, aS1.a), vadd(aS0.b, aS1.b), vadd(bS0.a, bS1.a), vadd(bS0.b, bS1.b)};
        const V SN[4] = {vadd(aN0.a, aN1.a), vadd(aN0.b, aN1.b), vadd(bN0.a, bN1.a), vadd(bN0.b, bN1.b)};
#pragma unroll
        for (int k = 0; k < 4; ++k) t2[k] = vpair(SP[k].y - SS[k].y, SN[k].x - SP[k].x);
        face_flux<V, true, AI, STD>(K, vmul(vlit<V>(0.5), vadd(a0.a, a1.a)), vadd(c0.a, c1.a), vadd(c0.b, c1.b),
                               vadd(d0, d1), n, t1, t2, Fc, Fd);
    };
    // single faces (the tile's low x and low y edges, the z face below the chunk)
    auto xface = [&](int am, int a0, int ap, int c0, int d0, int hL, int rL, V& Fc, V& Fd) {
        const Q* A0 = sA + a0;
        const Q* AM = sA + am;
        const Q* AP = sA + ap;
        const Q* B0 = sB + a0;
        const Q* BM = sB + am;
        const Q* BP = sB + ap;
        const Q* C0 = sC + c0;
        const V* D0 = sD + d0;
        const int hR = hL + 1;
        xface_core(A0[hL], B0[hL], A0[hR], B0[hR], A0[hL - HX], B0[hL - HX], A0[hR - HX], B0[hR - HX], A0[hL + HX],
                   B0[hL + HX], A0[hR + HX], B0[hR + HX], AP[hL], BP[hL], AP[hR], BP[hR], AM[hL], BM[hL], AM[hR],
                   BM[hR], C0[hL], C0[hR], D0[rL], D0[rL + 1], Fc, Fd);
    };
    auto yface = [&](int am, int a0, int ap, int c0, int d0, int hL, int rL, V& Fc, V& Fd) {
        const Q* A0 = sA + a0;
        const Q* AM = sA + am;
        const Q* AP = sA + ap;
        const Q* B0 = sB + a0;
        const Q* BM = sB + am;
        const Q* BP = sB + ap;
        const Q* C0 = sC + c0;
        const V* D0 = sD + d0;
        const int hN = hL + HX;
        yface_core(A0[hL], B0[hL], A0[hN], B0[hN], A0[hL + 1], B0[hL + 1], A0[hL - 1], B0[hL - 1], A0[hN + 1],
                   B0[hN + 1], A0[hN - 1], B0[hN - 1], AP[hL], BP[hL], AM[hL], BM[hL], AP[hN], BP[hN], AM[hN],
                   BM[hN], C0[hL], C0[hN], D0[rL], D0[rL + RX], Fc, Fd);
    };
    auto zface = [&](int z, int h, int r, V& Fc, V& Fd) {
        const Q* A0 = sA + (z & 3) * HP;
        const Q* A1 = sA + ((z + 1) & 3) * HP;
        const Q* B0 = sB + (z & 3) * HP;
        const Q* B1 = sB + ((z + 1) & 3) * HP;
        const Q* C0 = sC + slot3(z) * HP;
        const Q* C1 = sC + slot3(z + 1) * HP;
        const V* D0 = sD + (z & 1) * RP;
        const V* D1 = sD + ((z + 1) & 1) * RP;
        zface_core(A0[h], B0[h], A1[h], B1[h], A0[h + 1], B0[h + 1], A0[h - 1], B0[h - 1], A1[h + 1], B1[h + 1],
                   A1[h - 1], B1[h - 1], A0[h - HX], B0[h - HX], A1[h - HX], B1[h - HX], A0[h + HX], B0[h + HX],
                   A1[h + HX], B1[h + HX], C0[h], C1[h], D0[r], D1[r], Fc, Fd);
    };
    // the own pair's x, y and z faces on plane z: 32 records of {phi, Y} and
    // {mu_s, mu_l}, 4 of {c_s, c_l} and 4 rates, each read once
    auto own_faces = [&](int am, int a0, int ap, int c0, int c1, int d0, const V rate_here, const V rate_up,
                         V& phi_here, V& Fxc, V& Fxd, V& Fyc, V& Fyd, V& Fzc, V& Fzd) {
        const int h = own_h, r = own_r;
        const Q* A0 = sA + a0;
        const Q* AM = sA + am;
        const Q* AP = sA + ap;
        const Q* B0 = sB + a0;
        const Q* BM = sB + am;
        const Q* BP = sB + ap;
        const Q* C0 = sC + c0;
        const V* D0 = sD + d0;
        // plane z: the pair O, its x neighbours E, W, the pairs N, S and NE, SE, NW
        const Q aO = A0[h], bO = B0[h], aE = A0[h + 1], bE = B0[h + 1], aW = A0[h - 1], bW = B0[h - 1];
        const Q aN = A0[h + HX], bN = B0[h + HX], aS = A0[h - HX], bS = B0[h - HX];
        const Q aNE = A0[h + HX + 1], bNE = B0[h + HX + 1];
        // plane z+1 (U) and z-1 (D)
        const Q aU = AP[h], bU = BP[h], aUE = AP[h + 1], bUE = BP[h + 1], aUN = AP[h + HX], bUN = BP[h + HX];
        const Q aD = AM[h], bD = BM[h];
        const Q cO = C0[h];
        const V dO = rate_here;
        phi_here = aO.a;
        xface_core(aO, bO, aE, bE, aS, bS, A0[h - HX + 1], B0[h - HX + 1], aN, bN, aNE, bNE, aU, bU, aUE, bUE, aD,
                   bD, AM[h + 1], BM[h + 1], cO, C0[h + 1], dO, D0[r + 1], Fxc, Fxd);
        yface_core(aO, bO, aN, bN, aE, bE, aW, bW, aNE, bNE, A0[h + HX - 1], B0[h + HX - 1], aU, bU, aD, bD, aUN,
                   bUN, AM[h + HX], BM[h + HX], cO, C0[h + HX], dO, D0[r + RX], Fyc, Fyd);
        zface_core(aO, bO, aU, bU, aE, bE, aW, bW, aUE, bUE, AP[h - 1], BP[h - 1], aS, bS, AP[h - HX], BP[h - HX],
                   aN, bN, aUN, bUN, cO, sC[c1 + h], dO, rate_up, Fzc, Fzd);
    };
    auto z_noflux = [&](int z) {
        return (z == -1 && G.bc_lo[2] == BC_NOFLUX) || (z == nz - 1 && G.bc_hi[2] == BC_NOFLUX);
    };

    const int z0 = (zbase + (int)blockIdx.z) * zchunk;   // this CTA's chunk of planes
    const int z1 = min(nz, z0 + zchunk);
    if (z0 >= z1) return;

    // prologue: planes z0-2 .. z0+1 into the rings, rates of z0-1 and z0, the
    // z face (z0-1, z0).  The single staging slot is refilled only after a
    // barrier has ordered every read of it.
    for (int z = z0 - 2; z <= z0; ++z) {
        fetch(z, true, -1);
        fetched();
        store_plane(offA(z), offC(z));
        __syncthreads();
    }
    rates_plane(z0 - 1);
    fetch(z0 + 1, true, -1);
    fetched();
    __syncthreads();   // plane z0+1 reuses the {c_s, c_l} / phi slots of z0-2
    store_plane(offA(z0 + 1), offC(z0 + 1));
    __syncthreads();
    rates_plane(z0);
    fetch(z0 + 2, true, -1);
    V fzc_down, fzd_down;
    zface(z0 - 1, own_h, own_r, fzc_down, fzd_down);
    if (z_noflux(z0 - 1)) fzc_down = fzd_down = vpair(T(0), T(0));
    __syncthreads();   // the loop's first store reuses the {c_s, c_l} slot of z0-1

    // fluxes of the plane being updated, carried from its faces phase to its update
    V fxc = vlit<V>(0.0), fxd = fxc, fyc = fxc, fyd = fxc, fzc = fxc, fzd = fxc;
    // FP32: the own pair's rate and phi carried in registers from the plane
    // loop to the update (the rate of plane k is computed while plane k-1 is
    // faced, read by the z face of k and by the update of k)
    V rate_k = sD[(z0 & 1) * RP + own_r], rate_prev = fxc, phi_prev = fxc;
    // update of plane k from its fluxes and the own-cell state staged in sO
    // ring offsets of the planes an iteration k touches, rotated per plane:
    // A/B rings k-1 .. k+2, C/P rings k .. k+2, rates k, k+1
    int ra_m1 = offA(z0 - 1), ra_0 = offA(z0), ra_p1 = offA(z0 + 1), ra_p2 = offA(z0 + 2);
    int rc_0 = offC(z0), rc_p1 = offC(z0 + 1), rc_p2 = offC(z0 + 2);
    int rd_0 = offD(z0), rd_p1 = offD(z0 + 1);
    // update of plane k: its rate and phi sit at D offset rd_p1 and A offset
    // ra_m1 whenever it runs (inside iteration k+1, and after the loop)
    auto update = [&](int k) {
        const Q left = sFx[ty * FXP + tx];
        const V below = sFy[ty * TX + tx];
        const T bc_ = below.x, bd_ = below.y;
        const V dFc = vadd(vadd(vsub(fxc, left.a), vpair(fyc.x - bc_, fyc.y - fyc.x)), vsub(fzc, fzc_down));
        const V dFd = vadd(vadd(vsub(fxd, left.b), vpair(fyd.x - bd_, fyd.y - fyd.x)), vsub(fzd, fzd_down));
        const V c_k = vpair(own_state(0, 0), own_state(0, 1)), d_k = vpair(own_state(1, 0), own_state(1, 1));
        V phi_new;
        if constexpr (sizeof(T) == 4) phi_new = vfma(K.dt_dx2, rate_prev, phi_prev);
        else phi_new = vfma(K.dt_dx2, sD[rd_p1 + own_r], sA[ra_m1 + own_h].a);
        const V d_new = vfma(K.dt_dx2, dFd, d_k);
        const V dcv = vmul(K.dt_dx2, dFc);
        V c_new, lo_new;
        if constexpr (sizeof(T) == 4) {
            // compensated (TwoSum) update of c = hi + lo
            const V lo_k = vpair(own_state(2, 0), own_state(2, 1));
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
        if constexpr (TMA) {
            // into the out tile (rows y, y+1 of the pair); thread 0 stores the
            // tile's boxes after the next barrier (cells outside the grid are
            // clipped by the store)
            T* w = sW + (2 * ty) * TX + tx;
            w[0] = phi_new.x;
            w[TX] = phi_new.y;
            w[TX * TY] = c_new.x;
            w[TX * TY + TX] = c_new.y;
            w[2 * TX * TY] = d_new.x;
            w[2 * TX * TY + TX] = d_new.y;
            w[3 * TX * TY] = lo_new.x;
            w[3 * TX * TY + TX] = lo_new.y;
            fence_proxy_async_smem();   // before the asynchronous proxy reads the tile
        } else {
            const long long gi = (long long)k * sz + own_xy;
            if (in_lo) {
                phi_out[gi] = phi_new.x;
                c_out[gi] = c_new.x;
                d_out[gi] = d_new.x;
                if constexpr (sizeof(T) == 4) clo_out[gi] = lo_new.x;
            }
            if (in_hi) {
                phi_out[gi + nx] = phi_new.y;
                c_out[gi + nx] = c_new.y;
                d_out[gi + nx] = d_new.y;
                if constexpr (sizeof(T) == 4) clo_out[gi + nx] = lo_new.y;
            }
        }
        fzc_down = fzc;
        fzd_down = fzd;
    };
    // thread 0: the out tile of plane k to global memory (after a barrier that
    // follows the update), one box per state word
    auto store_tile = [&](int k) {
        if constexpr (TMA) {
            if (tid == 0) {
                tma_store_3d(&tw_phi, sW, x0, y0, k + zpad);
                tma_store_3d(&tw_c, sW + TX * TY, x0, y0, k + zpad);
                tma_store_3d(&tw_d, sW + 2 * TX * TY, x0, y0, k + zpad);
                tma_store_3d(&tw_clo, sW + 3 * TX * TY, x0, y0, k + zpad);
                bulk_commit();
            }
        }
    };

    // two phases per plane:
    //   1: update(k-1) | plane k+2 from staging into the rings
    //   2: copies of plane k+3 and of the own state of k in flight | rates of
    //      plane k+1 (a thread's faces read only its own new rate) | faces of k
    for (int k = z0; k < z1; ++k) {
        fetched();
        if (k > z0) update(k - 1);
        store_plane(ra_p2, rc_p2);
        __syncthreads();
        if (k > z0) store_tile(k - 1);
        fetch(k + 3, k + 1 < z1, k);
        const bool ghost_up = ghost(k + 1);
        if constexpr (sizeof(T) == 4) {
            // The own rate of plane k+1 goes to the z face in a register and to
            // shared memory only after the faces: with no shared store between
            // them, the records the rate and the faces both read are read once.
            const V rate_up = rate_of(ghost_up, ra_0, ra_p1, ra_p2, rc_0, rc_p1, rc_p2, own_dsc, own_xc);
            V phi_k;
            own_faces(ra_m1, ra_0, ra_p1, rc_0, rc_p1, rd_0, rate_k, rate_up, phi_k, fxc, fxd, fyc, fyd, fzc, fzd);
            sD[rd_p1 + own_r] = rate_up;
            if (bor_r >= 0)
                sD[rd_p1 + bor_r] = rate_of(ghost_up, ra_0, ra_p1, ra_p2, rc_0, rc_p1, rc_p2, bor_dsc, bor_xc);
            rate_prev = rate_k;
            phi_prev = phi_k;
            rate_k = rate_up;
        } else {   // FP64: one face at a time keeps fewer registers live
            sD[rd_p1 + own_r] = rate_of(ghost_up, ra_0, ra_p1, ra_p2, rc_0, rc_p1, rc_p2, own_dsc, own_xc);
            if (bor_r >= 0)
                sD[rd_p1 + bor_r] = rate_of(ghost_up, ra_0, ra_p1, ra_p2, rc_0, rc_p1, rc_p2, bor_dsc, bor_xc);
            xface(ra_m1, ra_0, ra_p1, rc_0, rd_0, own_h, own_r, fxc, fxd);
            yface(ra_m1, ra_0, ra_p1, rc_0, rd_0, own_h, own_r, fyc, fyd);
            zface(k, own_h, own_r, fzc, fzd);
        }
        if (nf_x) fxc = fxd = vpair(T(0), T(0));
        fyc = vmask(fyc, nf_ylo, nf_yhi);
        fyd = vmask(fyd, nf_ylo, nf_yhi);
        if (z_noflux(k)) fzc = fzd = vpair(T(0), T(0));
        sFx[ty * FXP + tx + 1] = Q{fxc, fxd};
        sFy[(ty + 1) * TX + tx] = vpair(fyc.y, fyd.y);
        if (tid < TYP) {
            // x faces on the tile's low x edge, pair row tid
            V ec, ed;
            xface(ra_m1, ra_0, ra_p1, rc_0, rd_0, (tid + 1) * HX + 1, (tid + 1) * RX, ec, ed);
            if (nf_x_edge) ec = ed = vpair(T(0), T(0));
            sFx[tid * FXP] = Q{ec, ed};
        } else if (tid >= 128 && tid < 128 + TX) {
            // y face on the tile's low y edge (upper lane of the pair row below the
            // tile), on warp 4: warps w and w + 4 share a scheduler, and warps 5-7
            // carry the ring's border rates, so both edge tasks go to the pair
            // (0, 4) that has no border rate (measured 1.1 % faster than warp 1)
            const int ex = tid - 128;
            V ec, ed;
            yface(ra_m1, ra_0, ra_p1, rc_0, rd_0, ex + 2, ex + 1, ec, ed);
            sFy[ex] = nf_y_edge ? vpair(T(0), T(0)) : vpair(ec.y, ed.y);
        }
        // the next update rewrites the out tile: its stores must have read it
        if constexpr (TMA)
            if (tid == 0) bulk_wait_read();
        __syncthreads();
        // rotate the ring offsets to iteration k+1
        const int ta = ra_m1;
        ra_m1 = ra_0; ra_0 = ra_p1; ra_p1 = ra_p2; ra_p2 = ta;
        const int tc = rc_0;
        rc_0 = rc_p1; rc_p1 = rc_p2; rc_p2 = tc;
        const int td = rd_0;
        rd_0 = rd_p1; rd_p1 = td;
    }
    fetched();
    update(z1 - 1);
    if constexpr (TMA) {
        __syncthreads();
        store_tile(z1 - 1);
        if (tid == 0) bulk_wait_all();
        // a wait that ran out: give copies still in flight a bounded time to
        // land before the CTA's shared memory is released
        if (tid == 0 && timed_out) mbar_wait_bounded(bar, stuck);
    }
}

// planes per CTA: minimise (waves of resident CTAs) x (planes + prologue) over
// the number of z chunks, so that small grids still fill every SM
static int choose_zchunk(long long tiles, int nz, long long resident) {
    int best = nz;
    double best_cost = 1e300;
    for (int chunks = 1; chunks <= std::max(1, nz / 8); ++chunks) {
        const int zc = (nz + chunks - 1) / chunks;
        const long long nch = (nz + zc - 1) / zc;
        const long long waves = (tiles * nch + resident - 1) / resident;
        const double cost = (double)waves * (zc + 3.0);
        if (cost < best_cost) {
            best_cost = cost;
            best = zc;
        }
    }
    return best;
}

template <typename T>
using Step3dKernel = decltype(&step3d_kernel<T, 32, 16, true, true, false, false>);

// the instances: [default physics][19-point Laplacian][a != 0], staged by TMA
// (FP32 only) or by per-cell copies
template <typename T, bool TMA>
static void step3d_table(Step3dKernel<T> k[2][2][2]) {
    constexpr int TX = 32, TY = 16;
    constexpr bool M = TMA && sizeof(T) == 4;
    k[0][0][0] = step3d_kernel<T, TX, TY, false, false, false, M>;
    k[0][0][1] = step3d_kernel<T, TX, TY, false, true, false, M>;
    k[0][1][0] = step3d_kernel<T, TX, TY, true, false, false, M>;
    k[0][1][1] = step3d_kernel<T, TX, TY, true, true, false, M>;
    k[1][0][0] = step3d_kernel<T, TX, TY, false, false, true, M>;
    k[1][0][1] = step3d_kernel<T, TX, TY, false, true, true, M>;
    k[1][1][0] = step3d_kernel<T, TX, TY, true, false, true, M>;
    k[1][1][1] = step3d_kernel<T, TX, TY, true, true, true, M>;
}

// kernel attributes (once per device) and the occupancy the z-chunking plans with
template <typename T>
static cudaError_t step3d_setup(int* per_sm, int* sms) {
    constexpr int TX = 32, TY = 16;
    using L = PTile<T, TX, TY>;
    static DeviceSetup setup;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= DeviceSetup::MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(setup.mu);
    if (!setup.done[dev]) {
        Step3dKernel<T> kt[2][2][2][2];
        step3d_table<T, false>(kt[0]);
        step3d_table<T, true>(kt[1]);
        // per-cell instances first: in FP64 the TMA table holds the same
        // functions, which then keep the larger limit
        for (int i = 0; i < 16 && e == cudaSuccess; ++i)
            e = cudaFuncSetAttribute((&kt[0][0][0][0])[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(i < 8 ? L::BYTES_CP : L::BYTES));
        if (e != cudaSuccess) return e;
        int s = 1, p = 1, q = 1;
        cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, kt[0][1][1][1], L::NT, L::BYTES_CP);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, kt[1][1][1][1], L::NT, L::BYTES);
        p = std::min(p, q);
        setup.sms[dev] = s;
        setup.per_sm[dev] = p < 1 ? 1 : p;
        setup.done[dev] = true;
    }
    *per_sm = setup.per_sm[dev];
    *sms = setup.sms[dev];
    return cudaSuccess;
}

template <typename T>
cudaError_t step3d_chunks(const HostProblem& P, int requested, int* zchunk, int* nchunks) {
    int per_sm = 1, sms = 1;
    cudaError_t e = step3d_setup<T>(&per_sm, &sms);
    if (e != cudaSuccess) return e;
    const long long tiles = ((P.n[0] + 31) / 32) * ((P.n[1] + 15) / 16);
    int zc = requested;
    if (zc <= 0) zc = choose_zchunk(tiles, (int)P.n[2], (long long)per_sm * sms);
    *zchunk = zc;
    *nchunks = (int)((P.n[2] + zc - 1) / zc);
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_step3d(const StepLaunch& a, const Consts<T>& C, const Clock<T>& Kc) {
    constexpr int TX = 32, TY = 16;
    using L = PTile<T, TX, TY>;
    // 19- or 7-point Laplacian x shape parameter a != 0 or a = 0
    // 19- or 7-point Laplacian x shape parameter a != 0 or a = 0 x default physics
    // (quintic h, M_i = D_i c_i: literal coefficients) or not
    const HostProblem& P = *a.prob;
    int zchunk = 0, nchunks = 0;
    cudaError_t e = step3d_chunks<T>(P, a.zchunk, &zchunk, &nchunks);
    if (e != cudaSuccess) return e;
    const PairConsts<typename L::V> K = make_pair_consts<T>(P, C);
    const GridConsts<T> G = make_grid_consts<T>(P, Kc);
    dim3 block(L::NT);
    dim3 grid((C.n[0] + TX - 1) / TX, (C.n[1] + TY - 1) / TY, 1);
    // all chunks, or chunks [zfirst, zfirst + zcount) only
    const int zfirst = a.zcount > 0 ? a.zfirst : 0;
    const int count = a.zcount > 0 ? std::min(a.zcount, nchunks - zfirst) : nchunks;
    if (count <= 0) return cudaSuccess;
    grid.z = count;
    // TMA plane loads (FP32): one tensor map per state word over planes -zpad
    // .. nz - 1 + zpad (a slab's arrays hold two ghost planes beyond each z
    // side) with the staging box.  Rows must be whole multiples of 16 bytes,
    // and a periodic x or y side, whose ghosts come from outside the box, takes
    // per-cell copies.
    CUtensorMap maps[8];   // inputs phi, c, d, c_lo (staging boxes), outputs (tile boxes)
    std::memset(maps, 0, sizeof(maps));
    int flags = 0;
    const int zpad = (P.bc_lo[2] == PF_BC_HALO || P.bc_hi[2] == PF_BC_HALO) ? 2 : 0;
    const bool periodic_xy = P.bc_lo[0] == PF_BC_PERIODIC || P.bc_hi[0] == PF_BC_PERIODIC ||
                             P.bc_lo[1] == PF_BC_PERIODIC || P.bc_hi[1] == PF_BC_PERIODIC;
    if (sizeof(T) == 4 && !a.no_tma && !periodic_xy && (P.n[0] * sizeof(T)) % 16 == 0) {
        const uint64_t n[3] = {(uint64_t)P.n[0], (uint64_t)P.n[1], (uint64_t)P.n[2] + 2 * zpad};
        const uint32_t box[3] = {(uint32_t)L::BXW, (uint32_t)L::BH, 1};
        const size_t plane = (size_t)P.n[0] * P.n[1] * sizeof(T);
        const uint32_t tile[3] = {(uint32_t)TX, (uint32_t)TY, 1};
        const void* src[8] = {a.phi_in, a.c_in, a.d_in, a.clo_in, a.phi_out, a.c_out, a.d_out, a.clo_out};
        bool ok = true;
        for (int f = 0; f < 8 && ok; ++f) {
            const char* base = static_cast<const char*>(src[f]) - zpad * plane;
            ok = reinterpret_cast<uintptr_t>(base) % 16 == 0 &&
                 encode_tensor_map_3d(&maps[f], sizeof(T) == 8, base, n, f < 4 ? box : tile);
        }
        if (ok) flags |= 1;
    }
    if (a.drop_copies) flags |= 2;
    Step3dKernel<T> kt[2][2][2];
    if (flags & 1) step3d_table<T, true>(kt);
    else step3d_table<T, false>(kt);
    const bool std_phys = P.interp == 0 && P.mobility == 0;
    auto kern = kt[std_phys ? 1 : 0][C.lap == 19 ? 1 : 0][P.a != 0.0 ? 1 : 0];
    kern<<<grid, block, (flags & 1) ? L::BYTES : L::BYTES_CP, a.stream>>>(
        static_cast<const T*>(a.phi_in), static_cast<const T*>(a.c_in), static_cast<const T*>(a.d_in),
        static_cast<const T*>(a.clo_in), static_cast<T*>(a.phi_out), static_cast<T*>(a.c_out),
        static_cast<T*>(a.d_out), static_cast<T*>(a.clo_out), K, G, zchunk, zfirst, maps[0], maps[1], maps[2],
        maps[3], maps[4], maps[5], maps[6], maps[7], flags, zpad, a.err);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled, looked up from the driver once per process
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

bool encode_tensor_map_3d(CUtensorMap* map, bool fp64, const void* base, const uint64_t n[3],
                          const uint32_t box[3]) {
    EncodeTiledFn fn = encoder();
    if (!fn) return false;
    const size_t es = fp64 ? 8 : 4;
    const cuuint64_t dims[3] = {n[0], n[1], n[2]};
    const cuuint64_t strides[2] = {n[0] * es, n[0] * n[1] * es};
    const cuuint32_t bdim[3] = {box[0], box[1], box[2]};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
              const_cast<void*>(base), dims, strides, bdim, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template cudaError_t launch_step3d<float>(const StepLaunch&, const Consts<float>&, const Clock<float>&);
template cudaError_t launch_step3d<double>(const StepLaunch&, const Consts<double>&, const Clock<double>&);
template cudaError_t step3d_chunks<float>(const HostProblem&, int, int*, int*);
template cudaError_t step3d_chunks<double>(const HostProblem&, int, int*, int*);

}  // namespace pf
