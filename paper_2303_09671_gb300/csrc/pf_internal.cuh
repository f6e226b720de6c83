// pf_internal.cuh -- device-side parameter block, boundary mapping and the
// pointwise functions of the phase-field model (arXiv 2303.09671), shared by
// the step and diagnostics kernels of libpf.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pf {

enum { BC_NOFLUX = 0, BC_PERIODIC = 1, BC_DIRICHLET = 2, BC_HALO = 3 };

// map_coord's marker for a Dirichlet ghost.  A halo side (the z ends of a slab
// of a decomposed grid) maps its ghost planes to their own, negative or
// >= n, indices: the state arrays hold the two ghost planes beyond such a
// side, imported from the neighbouring slab.  So tests for a Dirichlet ghost
// along z compare with DIR_GHOST; along x and y, where no side is a halo, any
// negative result is one.
constexpr int DIR_GHOST = -0x7fffffff - 1;

// Parameters in the kernel's arithmetic type T.
template <typename T>
struct Consts {
    int dim;
    int n[3];
    int bc_lo[3], bc_hi[3];
    int interp;     // 0 quintic, 1 cubic
    int lap;        // 3, 5, 9, 7, 19
    int mobility;   // 0 M = D c, 1 M = D
    T dir_phi, dir_cs, dir_cl;
    T dx, inv_dx, inv_2dx, inv_dx2;
    T H, sigma, inv_Mphi, D_s, D_l, log_ke, one_m_ke, A, one_m_A, b, a, delta2;
    T dt;
    // frozen temperature theta(x,t) = theta0 - G_theta * x_cell, with
    // theta0 = theta_ref + G_theta (x0 + v_pull t - shifts dx) folded on the host
    T G_theta;
    // h(phi) = phi^2 (h2 + phi (h3 + phi (h4 + phi h5))), h'(phi) = phi (dh1 +
    // phi (dh2 + phi (dh3 + phi dh4))) and M_i = Mi_c c_i + Mi_0, filled by
    // set_coefficients() from interp and mobility, so the kernels need no branch
    T h2, h3, h4, h5, dh1, dh2, dh3, dh4;
    T Ms_c, Ms_0, Ml_c, Ml_0;
};

// quintic h = 10 phi^3 - 15 phi^4 + 6 phi^5, cubic h = 3 phi^2 - 2 phi^3
// (the two choices of Sec. "Choice of interpolation functions"), and the
// mobility M_i = D_i c_i or the constant D_i
template <typename T>
__host__ __device__ inline void set_coefficients(Consts<T>& C) {
    const bool cubic = C.interp == 1;
    C.h2 = T(cubic ? 3 : 0);
    C.h3 = T(cubic ? -2 : 10);
    C.h4 = T(cubic ? 0 : -15);
    C.h5 = T(cubic ? 0 : 6);
    C.dh1 = T(cubic ? 6 : 0);
    C.dh2 = T(cubic ? -6 : 30);
    C.dh3 = T(cubic ? 0 : -60);
    C.dh4 = T(cubic ? 0 : 30);
    const bool cmob = C.mobility == 1;
    C.Ms_c = cmob ? T(0) : C.D_s;
    C.Ms_0 = cmob ? C.D_s : T(0);
    C.Ml_c = cmob ? T(0) : C.D_l;
    C.Ml_0 = cmob ? C.D_l : T(0);
}

// Per-launch time data.
template <typename T>
struct Clock {
    T theta0;   // see Consts::G_theta
};

// Map a possibly-ghost coordinate onto the interior (noflux: mirror about
// the boundary face; periodic: wrap; halo: the ghost plane itself, held in the
// state arrays); DIR_GHOST marks a Dirichlet ghost.  Cells further than the
// ghost width from the domain (only present in partial tiles, never used by
// interior cells) are clamped to keep loads in bounds.
__device__ __forceinline__ int map_coord(int i, int n, int lo, int hi) {
    if (i >= 0 && i < n) return i;
    int bc = (i < 0) ? lo : hi;
    int m;
    if (bc == BC_DIRICHLET) return DIR_GHOST;
    if (bc == BC_HALO) return i;
    if (bc == BC_PERIODIC) {
        m = i % n;
        if (m < 0) m += n;
        return m;
    }
    m = (i < 0) ? (-i - 1) : (2 * n - 1 - i);
    if (m < 0) m = 0;
    if (m > n - 1) m = n - 1;
    return m;
}

__device__ __forceinline__ float flog(float x) { return logf(x); }
__device__ __forceinline__ double flog(double x) { return log(x); }

// h(phi), p(phi) = h + a (phi - 1/2) phi^2 (1-phi)^2 (Eq. interpolation2), p'
template <typename T>
__device__ __forceinline__ T p_of(const Consts<T>& C, T f) {
    const T g = f * (T(1) - f);
    const T h = f * f * (C.h2 + f * (C.h3 + f * (C.h4 + f * C.h5)));
    return h + C.a * (f - T(0.5)) * g * g;
}
template <typename T>
__device__ __forceinline__ T dp_of(const Consts<T>& C, T f) {
    const T g = f * (T(1) - f);
    const T dh = f * (C.dh1 + f * (C.dh2 + f * (C.dh3 + f * C.dh4)));
    const T w = g * g;
    const T dw = T(2) * g * (T(1) - T(2) * f);
    return dh + C.a * (w + (f - T(0.5)) * dw);
}
template <typename T>
__device__ __forceinline__ T Ms_of(const Consts<T>& C, T cs) {
    return C.Ms_c * cs + C.Ms_0;
}
template <typename T>
__device__ __forceinline__ T Ml_of(const Consts<T>& C, T cl) {
    return C.Ml_c * cl + C.Ml_0;
}

}  // namespace pf
