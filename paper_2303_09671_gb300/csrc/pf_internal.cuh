// pf_internal.cuh -- device-side parameter block, boundary mapping and the
// pointwise functions of the phase-field model (arXiv 2303.09671), shared by
// the step and diagnostics kernels of libpf.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pf {

enum { BC_NOFLUX = 0, BC_PERIODIC = 1, BC_DIRICHLET = 2 };

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
};

// Per-launch time data.
template <typename T>
struct Clock {
    T theta0;   // see Consts::G_theta
};

// Map a possibly-ghost coordinate onto the interior (noflux: mirror about
// the boundary face; periodic: wrap); -1 marks a Dirichlet ghost.  Cells
// further than the ghost width from the domain (only present in partial
// tiles, never used by interior cells) are clamped to keep loads in bounds.
__device__ __forceinline__ int map_coord(int i, int n, int lo, int hi) {
    if (i >= 0 && i < n) return i;
    int bc = (i < 0) ? lo : hi;
    int m;
    if (bc == BC_DIRICHLET) return -1;
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
    T g = f * (T(1) - f);
    T h = (C.interp == 1) ? f * f * (T(3) - T(2) * f)
                          : f * f * f * (T(6) * f * f - T(15) * f + T(10));
    return h + C.a * (f - T(0.5)) * g * g;
}
template <typename T>
__device__ __forceinline__ T dp_of(const Consts<T>& C, T f) {
    T g = f * (T(1) - f);
    T dh = (C.interp == 1) ? T(6) * g : T(30) * g * g;
    T w = g * g;
    T dw = T(2) * g * (T(1) - T(2) * f);
    return dh + C.a * (w + (f - T(0.5)) * dw);
}
template <typename T>
__device__ __forceinline__ T Ms_of(const Consts<T>& C, T cs) {
    return C.mobility == 1 ? C.D_s : C.D_s * cs;
}
template <typename T>
__device__ __forceinline__ T Ml_of(const Consts<T>& C, T cl) {
    return C.mobility == 1 ? C.D_l : C.D_l * cl;
}

}  // namespace pf
