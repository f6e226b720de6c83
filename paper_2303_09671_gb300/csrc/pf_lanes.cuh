// pf_lanes.cuh -- two-lane arithmetic shared by the 3D and 2D step kernels
// (pf_step3d.cu, pf_step2d.cu): a thread owns the two cells (x, y) and
// (x, y+1) and evaluates them as one two-lane vector, in FP32 with the packed
// .f32x2 add/sub/mul/fma of sm_100-class GPUs (two FP32 operations per issue
// slot), in FP64 on double2 lanes.  Also: the face-flux algebra in grid units,
// p(phi) and p'(phi) on lanes, the lane-broadcast parameter blocks and the
// cp.async helpers.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include "pf_internal.cuh"
#include "pf_kernels.h"

namespace pf {

// ---------------------------------------------------------------- two lanes
template <typename T>
struct Lanes;
template <>
struct Lanes<float> {
    using V = float2;
};
template <>
struct Lanes<double> {
    using V = double2;
};

__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
    unsigned long long ra, rb, rr;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rr) : "l"(ra), "l"(rb));
    float2 r;
    memcpy(&r, &rr, 8);
    return r;
}
// FP32 reciprocal and natural logarithm from the PTX approximate instructions
// (rcp.approx, lg2.approx; flush-to-zero, as every operand here is a normal
// number of moderate size): 1/x to ~1 ulp, ln x = ln 2 log2 x to ~2^-22
// relative.  The FP64 path below is exact IEEE.
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ln_fast(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r * 0.693147180559945309f;
}
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(rcp_fast(a.x), rcp_fast(a.y)); }
__device__ __forceinline__ float2 vlog(float2 a) { return make_float2(ln_fast(a.x), ln_fast(a.y)); }
__device__ __forceinline__ float2 vpair(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 vrcp(double2 a) { return make_double2(1.0 / a.x, 1.0 / a.y); }
__device__ __forceinline__ double2 vlog(double2 a) { return make_double2(log(a.x), log(a.y)); }
__device__ __forceinline__ double2 vpair(double a, double b) { return make_double2(a, b); }

// a compile-time constant on both lanes
template <typename V>
__device__ __forceinline__ V vlit(double v);
template <>
__device__ __forceinline__ float2 vlit<float2>(double v) { return make_float2((float)v, (float)v); }
template <>
__device__ __forceinline__ double2 vlit<double2>(double v) { return make_double2(v, v); }

// two fields of a cell pair: one 16-byte shared-memory access in FP32
template <typename V>
struct alignas(2 * sizeof(V)) Q2 {
    V a, b;
};

// Parameters, each broadcast to both lanes (so that two-lane instructions
// can take them as operands), in grid units.  Pure numbers (1/2, 1/16, ...)
// are compile-time constants (vlit) instead: measured 1.3 % faster in 3D.
template <typename V>
struct PairConsts {
    V h2, h3, h4, h5, dh1, dh2, dh3, dh4, a_int;
    V Ms_c, Ms_0, Ml_c, Ml_0, b, A, one_m_A, one_m_ke, log_ke;
    V Ms_c_half, Ml_c_half, quarter_one_m_A;   // for face sums in place of face means
    V sigma, H, dx2, inv_Mphi, K_anti, delta2_dx2, delta2_4dx2, dt_dx2;
};

// Grid, boundaries, frozen temperature and the Dirichlet ghost state.
template <typename T>
struct GridConsts {
    int n[3], bc_lo[3], bc_hi[3];
    T dx, theta0, G_theta;
    T dir_phi, dir_c, dir_d;   // ghost phi and its c = p c_s + (1-p) c_l, d = c_s - c_l
};

// asynchronous global -> shared copies (cp.async, completion awaited per thread)
template <typename T>
__device__ __forceinline__ void cp_async(T* smem_dst, const T* gsrc) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// p(phi) of Eq. interpolation2 and its derivative, two lanes.  AI = false: the
// shape parameter a is 0 and p = h (the term a (phi - 1/2) phi^2 (1-phi)^2 is
// skipped, which leaves the result bit for bit the same)
// STD = true: the quintic h with its coefficients as literals (the same
// operations as the general form, whose zero terms drop out exactly)
template <bool AI = true, bool STD = false, typename V>
__device__ __forceinline__ V vp_of(const PairConsts<V>& K, V f) {
    const V h = STD ? vmul(vmul(f, f), vmul(f, vfma(f, vfma(f, vlit<V>(6.0), vlit<V>(-15.0)), vlit<V>(10.0))))
                    : vmul(vmul(f, f), vfma(f, vfma(f, vfma(f, K.h5, K.h4), K.h3), K.h2));
    if constexpr (!AI) return h;
    const V g = vmul(f, vsub(vlit<V>(1.0), f));
    return vfma(vmul(K.a_int, vsub(f, vlit<V>(0.5))), vmul(g, g), h);
}
template <bool AI = true, bool STD = false, typename V>
__device__ __forceinline__ V vdp_of(const PairConsts<V>& K, V f) {
    const V dh = STD ? vmul(f, vmul(f, vfma(f, vfma(f, vlit<V>(30.0), vlit<V>(-60.0)), vlit<V>(30.0))))
                     : vmul(f, vfma(f, vfma(f, vfma(f, K.dh4, K.dh3), K.dh2), K.dh1));
    if constexpr (!AI) return dh;
    const V g = vmul(f, vsub(vlit<V>(1.0), f));
    // d/dphi [g^2 (phi - 1/2)] = g^2 + 2 g (1 - 2 phi)(phi - 1/2) = g^2 - 4 g (phi - 1/2)^2
    const V s = vsub(f, vlit<V>(0.5));
    const V w = vmul(g, vsub(g, vmul(vlit<V>(4.0), vmul(s, s))));
    return vfma(K.a_int, w, dh);
}

// Fluxes through a face (dx times F_c, F_d of the model) from the face state:
// f = face mean of phi; cs2, cl2 = the sums (twice the face means) of c_s and
// c_l, taken by constants halved on the host (M_s = M_s_c c_s + M_s_0 becomes
// (M_s_c / 2) cs2 + M_s_0; exact, since halving is); pds = sum of the two
// cells' dx^2 phidot; n = the
// normal differences R - L of {phi, Y, mu_s, mu_l}; t1, t2 = the transverse
// sums of four centred differences (4 dx times the face's transverse
// gradient).  With T_i = M_i [n_i (|t|^2/16 + delta^2 dx^2) - n_phi (t.t_i)/16]
// and w_s + w_l = 1, p w_s - (1-p) w_l = a(phi) (Eq. shape_function):
//   F_c = r [q n_phi (n_phi n_Y + t.t_Y/16) + p T_s + (1-p) T_l + at a(phi)]
//   F_d = r [T_s - T_l + at],  at = (1-A) d phidot dx^2 n_phi,
//   r = 1/(n_phi^2 + |t|^2/16 + delta^2 dx^2)
// T2 = false: a face of a 2D grid, with one transverse direction (t2 unused)
template <typename V, bool T2 = true, bool AI = true, bool STD = false>
__device__ __forceinline__ void face_flux(const PairConsts<V>& K, V f, V cs2, V cl2, V pds, const V n[4],
                                          const V t1[4], const V t2[4], V& Fc, V& Fd) {
    const V d2 = vsub(cs2, cl2);   // twice the face d
    const V p = vp_of<AI, STD>(K, f);
    const V omp = vsub(vlit<V>(1.0), p);
    const V Ms = STD ? vmul(K.Ms_c_half, cs2) : vfma(K.Ms_c_half, cs2, K.Ms_0);
    const V Ml = STD ? vmul(K.Ml_c_half, cl2) : vfma(K.Ml_c_half, cl2, K.Ml_0);
    const V bMl = vmul(K.b, Ml);
    const V iMbar = vrcp(vfma(bMl, p, vmul(Ms, omp)));
    const V tt = T2 ? vfma(t1[0], t1[0], vmul(t2[0], t2[0])) : vmul(t1[0], t1[0]);
    const V gt2d = vfma(tt, vlit<V>(0.0625), K.delta2_dx2);
    const V r = vrcp(vfma(n[0], n[0], gt2d));
    const V m = vmul(n[0], vlit<V>(-0.0625));          // -n_phi / 16
    const V dY = vfma(T2 ? vfma(t1[0], t1[1], vmul(t2[0], t2[1])) : vmul(t1[0], t1[1]), vlit<V>(0.0625),
                      vmul(n[0], n[1]));
    const V ts = T2 ? vfma(t1[0], t1[2], vmul(t2[0], t2[2])) : vmul(t1[0], t1[2]);
    const V tl = T2 ? vfma(t1[0], t1[3], vmul(t2[0], t2[3])) : vmul(t1[0], t1[3]);
    const V Ts = vmul(Ms, vfma(m, ts, vmul(n[2], gt2d)));
    const V Tl = vmul(Ml, vfma(m, tl, vmul(n[3], gt2d)));
    const V at = vmul(vmul(K.quarter_one_m_A, pds), vmul(d2, n[0]));
    const V pomp = vmul(p, omp);
    const V q = vmul(vmul(Ms, Ml), vmul(vfma(K.b, p, omp), iMbar));
    const V afn = vmul(vsub(Ms, bMl), vmul(pomp, iMbar));
    V acc = vmul(vmul(q, n[0]), dY);
    acc = vfma(p, Ts, acc);
    acc = vfma(omp, Tl, acc);
    acc = vfma(at, afn, acc);
    Fc = vmul(r, acc);
    Fd = vmul(r, vadd(vsub(Ts, Tl), at));
}

// lane-wise zero
template <typename V>
__device__ __forceinline__ V vmask(V v, bool zero_lo, bool zero_hi) {
    if (zero_lo) v.x = 0;
    if (zero_hi) v.y = 0;
    return v;
}

// FP64 host value of p(phi) for the Dirichlet ghost state
inline double p_host3(const HostProblem& P, double f) {
    const double g = f * (1.0 - f);
    const double h = (P.interp == 1) ? f * f * (3.0 - 2.0 * f) : f * f * f * (6.0 * f * f - 15.0 * f + 10.0);
    return h + P.a * (f - 0.5) * g * g;
}

template <typename V, typename T>
inline V splat(double v) {
    V r;
    r.x = T(v);
    r.y = T(v);
    return r;
}

template <typename T>
inline PairConsts<typename Lanes<T>::V> make_pair_consts(const HostProblem& P, const Consts<T>& C) {
    using V = typename Lanes<T>::V;
    auto S = [](double v) { return splat<V, T>(v); };
    PairConsts<V> K;
    K.h2 = S(C.h2); K.h3 = S(C.h3); K.h4 = S(C.h4); K.h5 = S(C.h5);
    K.dh1 = S(C.dh1); K.dh2 = S(C.dh2); K.dh3 = S(C.dh3); K.dh4 = S(C.dh4);
    K.a_int = S(P.a);
    K.Ms_c = S(C.Ms_c); K.Ms_0 = S(C.Ms_0); K.Ml_c = S(C.Ml_c); K.Ml_0 = S(C.Ml_0);
    K.b = S(P.b); K.A = S(P.A); K.one_m_A = S(1.0 - P.A);
    K.Ms_c_half = S(0.5 * C.Ms_c); K.Ml_c_half = S(0.5 * C.Ml_c); K.quarter_one_m_A = S(0.25 * (1.0 - P.A));
    K.one_m_ke = S(1.0 - P.k_e); K.log_ke = S(std::log(P.k_e));
    const double dx2 = P.dx * P.dx;
    K.sigma = S(P.sigma); K.H = S(P.H); K.dx2 = S(dx2); K.inv_Mphi = S(1.0 / P.M_phi);
    K.K_anti = S((1.0 - P.A) * (1.0 - P.A) * P.b * 4.0 * dx2);
    K.delta2_dx2 = S(P.delta * P.delta * dx2);
    K.delta2_4dx2 = S(4.0 * P.delta * P.delta * dx2);
    K.dt_dx2 = S(P.dt / dx2);
    return K;
}

template <typename T>
inline GridConsts<T> make_grid_consts(const HostProblem& P, const Clock<T>& Kc) {
    GridConsts<T> G;
    for (int a = 0; a < 3; ++a) {
        G.n[a] = (int)P.n[a];
        G.bc_lo[a] = P.bc_lo[a];
        G.bc_hi[a] = P.bc_hi[a];
    }
    G.dx = T(P.dx);
    G.theta0 = Kc.theta0;
    G.G_theta = T(P.G_theta);
    const double pg = p_host3(P, P.dir_phi);
    G.dir_phi = T(P.dir_phi);
    G.dir_c = T(pg * P.dir_cs + (1.0 - pg) * P.dir_cl);
    G.dir_d = T(P.dir_cs - P.dir_cl);
    return G;
}

}  // namespace pf
