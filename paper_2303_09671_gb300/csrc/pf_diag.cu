// pf_diag.cu -- FP64 diagnostics (discrete free energy, total solute, front,
// c_max), the 1D moving-window shift and the conversions between the
// caller's (phi, c_s, c_l) and the device state (phi, c, d[, c_lo]).
//
// Reductions are deterministic: a grid fixed by the problem size and the
// device (at most 8 blocks per SM, fewer for small grids, so that a 1D run does
// not launch a thousand idle blocks every step) writes one partial per block
// (warp-shuffle tree inside the block), and a single block sums the partials in
// a fixed order.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include "pf_internal.cuh"
#include "pf_kernels.h"

namespace pf {

static constexpr int DIAG_THREADS = 256;

size_t diag_scratch_doubles(const HostProblem&) { return 2 * (size_t)DIAG_MAX_BLOCKS; }

// largest grid of the reductions and conversions on the current device: 8
// blocks of 256 threads per SM (the SM count queried once per device), at most
// DIAG_MAX_BLOCKS
static int diag_grid() {
    static DeviceSetup setup;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= DeviceSetup::MAX_DEVICES) {
        cudaGetLastError();
        return DIAG_MAX_BLOCKS;
    }
    std::lock_guard<std::mutex> lock(setup.mu);
    if (!setup.done[dev]) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            sms = DIAG_MAX_BLOCKS / 8;
        }
        setup.value[dev] = (size_t)std::min(8 * sms, DIAG_MAX_BLOCKS);
        setup.done[dev] = true;
    }
    return (int)setup.value[dev];
}

// blocks for a grid-stride pass over `items`: one per 64 items up to
// diag_grid(), so that small FP64 problems spread their (slow) FP64 work over
// many SMs
static int diag_blocks(long long items) {
    const long long b = (items + 63) / 64;
    const long long cap = diag_grid();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

struct DiagConsts {
    int n[3], bc_lo[3], bc_hi[3], dim, lap, interp;
    double dir_phi, dx, H, sigma, k_e, a, theta0, G_theta, dV;
};

__device__ __forceinline__ double p_d(const DiagConsts& C, double f) {
    double g = f * (1.0 - f);
    double h = (C.interp == 1) ? f * f * (3.0 - 2.0 * f) : f * f * f * (6.0 * f * f - 15.0 * f + 10.0);
    return h + C.a * (f - 0.5) * g * g;
}

template <typename T>
__device__ __forceinline__ double fetch_phi(const DiagConsts& C, const T* phi, int i, int j, int k) {
    int mi = map_coord(i, C.n[0], C.bc_lo[0], C.bc_hi[0]);
    int mj = (C.dim >= 2) ? map_coord(j, C.n[1], C.bc_lo[1], C.bc_hi[1]) : 0;
    int mk = (C.dim >= 3) ? map_coord(k, C.n[2], C.bc_lo[2], C.bc_hi[2]) : 0;
    if (mi < 0 || mj < 0 || mk == DIR_GHOST) return C.dir_phi;
    return (double)phi[((long long)mk * C.n[1] + mj) * C.n[0] + mi];
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// block reduction of two values (sum or max), result valid in thread 0
template <bool MAX>
__device__ void block_reduce2(double& a, double& b) {
    __shared__ double sa[DIAG_THREADS / 32], sb[DIAG_THREADS / 32];
    a = MAX ? warp_max(a) : warp_sum(a);
    b = MAX ? warp_max(b) : warp_sum(b);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    if (l == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (w == 0) {
        a = (l < DIAG_THREADS / 32) ? sa[l] : (MAX ? -INFINITY : 0.0);
        b = (l < DIAG_THREADS / 32) ? sb[l] : (MAX ? -INFINITY : 0.0);
        a = MAX ? warp_max(a) : warp_sum(a);
        b = MAX ? warp_max(b) : warp_sum(b);
    }
}

// state accessors: c (with its FP32 low word), d -> c_s, c_l in FP64
template <typename T>
struct StateView {
    const T* phi;
    const T* c;
    const T* d;
    const T* clo;   // nullptr in FP64
    __device__ __forceinline__ double cval(long long i) const {
        return (double)c[i] + (clo ? (double)clo[i] : 0.0);
    }
    // total c, and (ENERGY) phi, p(phi), c_s, c_l of cell i
    template <bool ENERGY>
    __device__ __forceinline__ void cell(const DiagConsts& C, long long i, double& cc, double& f, double& p,
                                         double& s, double& l) const {
        cc = cval(i);
        if (!ENERGY) return;
        f = (double)phi[i];
        const double dd = (double)d[i];
        p = p_d(C, f);
        s = cc + (1.0 - p) * dd;
        l = cc - p * dd;
    }
};

// the caller's fields (phi, c_s, c_l) read directly (pf_energy_solute_noalloc)
template <typename T>
struct FieldView {
    const T* phi;
    const T* cs;
    const T* cl;
    template <bool ENERGY>
    __device__ __forceinline__ void cell(const DiagConsts& C, long long i, double& cc, double& f, double& p,
                                         double& s, double& l) const {
        f = (double)phi[i];
        s = (double)cs[i];
        l = (double)cl[i];
        p = p_d(C, f);
        cc = p * s + (1.0 - p) * l;   // Eq. model1 with g = p
    }
};

template <typename View, bool ENERGY>
__global__ void __launch_bounds__(DIAG_THREADS)
energy_solute_kernel(View S, DiagConsts C, double* __restrict__ part) {
    const long long N = (long long)C.n[0] * C.n[1] * C.n[2];
    double eF = 0.0, eS = 0.0;
    const double one_m_ke = 1.0 - C.k_e, log_ke = log(C.k_e);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        double cc, f = 0.0, p = 0.0, s = 0.0, l = 0.0;
        S.template cell<ENERGY>(C, c, cc, f, p, s, l);
        eS += cc;
        if (!ENERGY) continue;
        const int i = (int)(c % C.n[0]);
        const int j = (int)((c / C.n[0]) % C.n[1]);
        const int k = (int)(c / ((long long)C.n[0] * C.n[1]));
        const double theta = C.theta0 - C.G_theta * (((double)i + 0.5) * C.dx);
        const double fs = -one_m_ke * theta + s * (log(s) - log_ke - 1.0);
        const double fl = l * (log(l) - 1.0);
        const double fdw = f * f * (1.0 - f) * (1.0 - f);
        // gradient energy: each stencil pair once, weights of the Laplacian
        double gs = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int nzc = (dx != 0) + (dy != 0) + (dz != 0);
                    if (nzc == 0) continue;
                    double w = 0.0;
                    if (C.lap == 3) w = (dy == 0 && dz == 0) ? 1.0 : 0.0;
                    else if (C.lap == 5) w = (dz == 0 && nzc == 1) ? 1.0 : 0.0;
                    else if (C.lap == 9) w = (dz != 0) ? 0.0 : (nzc == 1 ? 2.0 / 3.0 : 1.0 / 6.0);
                    else if (C.lap == 7) w = (nzc == 1) ? 1.0 : 0.0;
                    else w = (nzc == 1) ? 1.0 / 3.0 : (nzc == 2 ? 1.0 / 6.0 : 0.0);
                    if (w == 0.0) continue;
                    const double dphi = fetch_phi(C, S.phi, i + dx, j + dy, k + dz) - f;
                    gs += w * dphi * dphi;
                }
        eF += C.H * fdw + p * fs + (1.0 - p) * fl + 0.5 * C.sigma * 0.5 * gs / (C.dx * C.dx);
    }
    block_reduce2<false>(eF, eS);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = eF;
        part[gridDim.x + blockIdx.x] = eS;
    }
}

// out[0..1] = the two sums; with `slot`, out[2 k..2 k+1] for k = *slot, then
// *slot = k + 1 (a record written from a replayed graph)
__global__ void __launch_bounds__(DIAG_THREADS)
finish_sum2(const double* __restrict__ part, int nb, double scale, double* __restrict__ out,
            long long* __restrict__ slot) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += part[i];
        b += part[nb + i];
    }
    block_reduce2<false>(a, b);
    if (threadIdx.x == 0) {
        long long k = 0;
        if (slot != nullptr) {
            k = *slot;
            *slot = k + 1;
        }
        out[2 * k] = a * scale;
        out[2 * k + 1] = b * scale;
    }
}

template <typename T>
__global__ void __launch_bounds__(DIAG_THREADS)
front_kernel(StateView<T> S, DiagConsts C, double* __restrict__ part) {
    const long long rows = (long long)C.n[1] * C.n[2];
    double xf = -INFINITY, cm = -INFINITY;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        const T* prow = S.phi + r * C.n[0];
        for (int i = C.n[0] - 2; i >= 0; --i) {
            const double a = (double)prow[i], b = (double)prow[i + 1];
            if (a >= 0.5 && b < 0.5) {
                xf = fmax(xf, ((double)i + 0.5 + (a - 0.5) / (a - b)) * C.dx);
                break;
            }
        }
        for (int i = 0; i < C.n[0]; ++i) cm = fmax(cm, S.cval(r * C.n[0] + i));
    }
    block_reduce2<true>(xf, cm);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = xf;
        part[gridDim.x + blockIdx.x] = cm;
    }
}

__global__ void __launch_bounds__(DIAG_THREADS)
finish_max2(const double* __restrict__ part, int nb, double* __restrict__ out) {
    double a = -INFINITY, b = -INFINITY;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a = fmax(a, part[i]);
        b = fmax(b, part[nb + i]);
    }
    block_reduce2<true>(a, b);
    if (threadIdx.x == 0) {
        out[0] = (a == -INFINITY) ? NAN : a;
        out[1] = b;
    }
}

// store an FP64 value of c as the state's c (and low word in FP32)
template <typename T>
__device__ __forceinline__ void put_c(T* c, T* clo, long long i, double v) {
    const T hi = (T)v;
    c[i] = hi;
    if (clo) clo[i] = (T)(v - (double)hi);
}

template <typename T>
__global__ void shift_kernel(StateView<T> in, const T* plo_in, T* po, T* co, T* dout, T* clo_out,
                             T* plo_out, int n, double fphi, double fc, double fd) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < n - 1) {
            po[i] = in.phi[i + 1];
            co[i] = in.c[i + 1];
            dout[i] = in.d[i + 1];
            if (clo_out) clo_out[i] = in.clo[i + 1];
            if (plo_out) plo_out[i] = plo_in[i + 1];
        } else {
            po[i] = (T)fphi;
            dout[i] = (T)fd;
            put_c(co, clo_out, i, fc);
            if (plo_out) plo_out[i] = (T)(fphi - (double)(T)fphi);
        }
    }
}

template <typename T>
__global__ void to_state_kernel(const T* __restrict__ phi, const T* __restrict__ cs,
                                const T* __restrict__ cl, long long n, DiagConsts C, T* po,
                                T* co, T* dout, T* clo) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double f = (double)phi[i], s = (double)cs[i], l = (double)cl[i];
        const double p = p_d(C, f);
        po[i] = phi[i];
        put_c(co, clo, i, p * s + (1.0 - p) * l);
        dout[i] = (T)(s - l);
    }
}

// FP32 input: the conversion in FP32 arithmetic (the FP64 units of a GB300
// are a small fraction of its FP32 rate).  p(phi) is evaluated in FP32 and
// c = c_l + p (c_s - c_l) is kept exactly as an unevaluated sum hi + lo of
// two floats: c_s - c_l and c_l + p d by TwoSum, p d by an FMA-based exact
// product (Knuth; Dekker), so the stored (c, c_lo) carries ~2^-48 relative
// error with respect to that p.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// one cell: (phi, c_s, c_l) -> (c, c_lo, d)
__device__ __forceinline__ void convert_f32(float f, float s, float l, float a, bool cubic, float& c,
                                            float& clo, float& d) {
    const float g = f * (1.0f - f);
    const float h = cubic ? f * f * (3.0f - 2.0f * f) : f * f * f * (f * (6.0f * f - 15.0f) + 10.0f);
    const float p = h + a * (f - 0.5f) * g * g;
    float dh, dl;
    two_sum(s, -l, dh, dl);
    const float prod = p * dh;
    const float small = fmaf(p, dl, fmaf(p, dh, -prod));
    float hi, e;
    two_sum(l, prod, hi, e);
    const float lo = e + small;
    c = hi + lo;
    clo = lo - (c - hi);
    d = dh;
}

__global__ void __launch_bounds__(DIAG_THREADS)
to_state_f32_kernel(const float* __restrict__ phi, const float* __restrict__ cs,
                    const float* __restrict__ cl, long long n, DiagConsts C, float* __restrict__ po,
                    float* __restrict__ co, float* __restrict__ dout, float* __restrict__ clo,
                    float* __restrict__ plo) {
    const float a = (float)C.a;
    const bool cubic = C.interp == 1;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float f = phi[i];
        float c, lo, d;
        convert_f32(f, cs[i], cl[i], a, cubic, c, lo, d);
        po[i] = f;
        if (plo) plo[i] = 0.0f;
        co[i] = c;
        clo[i] = lo;
        dout[i] = d;
    }
}

// The same with 16-byte loads and stores, 4 cells per thread and iteration,
// for 16-byte aligned arrays (the conversion from host memory is bound by the
// link, and wide requests keep more bytes in flight per thread); cells
// [4 (n / 4), n) are left to the scalar kernel.
__global__ void __launch_bounds__(DIAG_THREADS)
to_state_f32x4_kernel(const float4* __restrict__ phi, const float4* __restrict__ cs,
                      const float4* __restrict__ cl, long long n4, DiagConsts C, float4* __restrict__ po,
                      float4* __restrict__ co, float4* __restrict__ dout, float4* __restrict__ clo,
                      float4* __restrict__ plo) {
    const float a = (float)C.a;
    const bool cubic = C.interp == 1;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 f = phi[i], s = cs[i], l = cl[i];
        float4 c, lo, d;
        convert_f32(f.x, s.x, l.x, a, cubic, c.x, lo.x, d.x);
        convert_f32(f.y, s.y, l.y, a, cubic, c.y, lo.y, d.y);
        convert_f32(f.z, s.z, l.z, a, cubic, c.z, lo.z, d.z);
        convert_f32(f.w, s.w, l.w, a, cubic, c.w, lo.w, d.w);
        po[i] = f;
        if (plo) plo[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        co[i] = c;
        clo[i] = lo;
        dout[i] = d;
    }
}

// FP32 conversion of cells [0, n): the wide kernel where every array is 16-byte
// aligned, the scalar kernel for the rest
static void to_state_f32(const float* phi, const float* cs, const float* cl, long long n, const DiagConsts& C,
                         float* po, float* co, float* dout, float* clo, float* plo, int blocks,
                         cudaStream_t s) {
    auto al = [](const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    long long n4 = 0;
    if (al(phi) && al(cs) && al(cl) && al(po) && al(co) && al(dout) && al(clo) && al(plo)) {
        n4 = n / 4;
        if (n4 > 0)
            to_state_f32x4_kernel<<<blocks, DIAG_THREADS, 0, s>>>(
                (const float4*)phi, (const float4*)cs, (const float4*)cl, n4, C, (float4*)po, (float4*)co,
                (float4*)dout, (float4*)clo, (float4*)plo);
    }
    const long long d = 4 * n4;
    if (d < n)
        to_state_f32_kernel<<<blocks, DIAG_THREADS, 0, s>>>(phi + d, cs + d, cl + d, n - d, C, po + d, co + d,
                                                            dout + d, clo + d, plo ? plo + d : nullptr);
}

// FP32 state: total of c = c_hi + c_lo.  Each thread accumulates its cells as
// a renormalised float pair (TwoSum), so the FP32 pipes do the work; the
// per-thread totals then enter the FP64 block reduction.  Deterministic: the
// cells of a thread and the reduction order are fixed.
__global__ void __launch_bounds__(DIAG_THREADS)
solute_f32_kernel(const float* __restrict__ c, const float* __restrict__ clo, long long n,
                  double* __restrict__ part) {
    float ah = 0.0f, al = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n4 = n / 4;
    const float4* c4 = reinterpret_cast<const float4*>(c);
    const float4* l4 = reinterpret_cast<const float4*>(clo);
    auto add = [&](float x, float y) {
        float s, e;
        two_sum(ah, x, s, e);
        const float t = al + (e + y);
        ah = s + t;
        al = t - (ah - s);
    };
    for (long long i = t0; i < n4; i += stride) {
        const float4 x = c4[i], y = l4[i];
        add(x.x, y.x);
        add(x.y, y.y);
        add(x.z, y.z);
        add(x.w, y.w);
    }
    for (long long i = 4 * n4 + t0; i < n; i += stride) add(c[i], clo[i]);
    double v = (double)ah + (double)al, unused = 0.0;
    block_reduce2<false>(v, unused);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = 0.0;
        part[gridDim.x + blockIdx.x] = v;
    }
}

template <typename T>
__global__ void from_state_kernel(StateView<T> S, long long n, DiagConsts C, T* phi, T* cs, T* cl) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double f = (double)S.phi[i], c = S.cval(i), d = (double)S.d[i];
        const double p = p_d(C, f);
        phi[i] = S.phi[i];
        cs[i] = (T)(c + (1.0 - p) * d);
        cl[i] = (T)(c - p * d);
    }
}

// FP32 state -> (phi, c_s, c_l) in FP32 arithmetic: p(phi) in FP32, then
// c_s = c_hi + fma(1 - p, d, c_lo), c_l = c_hi + fma(-p, d, c_lo), so that the
// low word of c enters before the one rounding of each result
__device__ __forceinline__ void from_f32(float f, float hi, float lo, float d, float a, bool cubic, float& s,
                                         float& l) {
    const float g = f * (1.0f - f);
    const float h = cubic ? f * f * (3.0f - 2.0f * f) : f * f * f * (f * (6.0f * f - 15.0f) + 10.0f);
    const float p = h + a * (f - 0.5f) * g * g;
    s = hi + fmaf(1.0f - p, d, lo);
    l = hi + fmaf(-p, d, lo);
}

__global__ void __launch_bounds__(DIAG_THREADS)
from_state_f32_kernel(const float* __restrict__ phi, const float* __restrict__ c, const float* __restrict__ clo,
                      const float* __restrict__ d, long long n, DiagConsts C, float* __restrict__ po,
                      float* __restrict__ cs, float* __restrict__ cl) {
    const float a = (float)C.a;
    const bool cubic = C.interp == 1;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float s, l;
        from_f32(phi[i], c[i], clo[i], d[i], a, cubic, s, l);
        po[i] = phi[i];
        cs[i] = s;
        cl[i] = l;
    }
}

// the same, 4 cells per thread and iteration with 16-byte accesses (every
// array 16-byte aligned): the read-back to page-locked host memory is bound by
// the host link, and wide requests keep more bytes in flight per thread
__global__ void __launch_bounds__(DIAG_THREADS)
from_state_f32x4_kernel(const float4* __restrict__ phi, const float4* __restrict__ c,
                        const float4* __restrict__ clo, const float4* __restrict__ d, long long n4, DiagConsts C,
                        float4* __restrict__ po, float4* __restrict__ cs, float4* __restrict__ cl) {
    const float a = (float)C.a;
    const bool cubic = C.interp == 1;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 f = phi[i], h = c[i], lo = clo[i], dd = d[i];
        float4 s, l;
        from_f32(f.x, h.x, lo.x, dd.x, a, cubic, s.x, l.x);
        from_f32(f.y, h.y, lo.y, dd.y, a, cubic, s.y, l.y);
        from_f32(f.z, h.z, lo.z, dd.z, a, cubic, s.z, l.z);
        from_f32(f.w, h.w, lo.w, dd.w, a, cubic, s.w, l.w);
        po[i] = f;
        cs[i] = s;
        cl[i] = l;
    }
}

static DiagConsts make_diag(const HostProblem& P, int64_t step, int64_t shifts) {
    DiagConsts C;
    for (int a = 0; a < 3; ++a) {
        C.n[a] = (int)P.n[a];
        C.bc_lo[a] = P.bc_lo[a];
        C.bc_hi[a] = P.bc_hi[a];
    }
    C.dim = P.dim;
    C.lap = P.lap;
    C.interp = P.interp;
    C.dir_phi = P.dir_phi;
    C.dx = P.dx;
    C.H = P.H;
    C.sigma = P.sigma;
    C.k_e = P.k_e;
    C.a = P.a;
    const double t = (double)step * P.dt;
    C.theta0 = P.theta_ref + P.G_theta * (P.x0 + P.v_pull * t - (double)shifts * P.dx);
    C.G_theta = P.G_theta;
    C.dV = std::pow(P.dx, P.dim);
    return C;
}

template <typename T>
static StateView<T> view(const Fields& f) {
    return StateView<T>{(const T*)f.phi, (const T*)f.c, (const T*)f.d, (const T*)f.clo};
}

cudaError_t launch_energy_solute(const HostProblem& P, const Fields& f, int64_t step,
                                 int64_t shifts, bool with_energy, double* scratch, double* out,
                                 cudaStream_t s, long long* slot) {
    const DiagConsts C = make_diag(P, step, shifts);
    const int nb = diag_blocks(P.cells());
    if (P.precision == 1) {
        if (with_energy)
            energy_solute_kernel<StateView<double>, true><<<nb, DIAG_THREADS, 0, s>>>(view<double>(f), C, scratch);
        else
            energy_solute_kernel<StateView<double>, false><<<nb, DIAG_THREADS, 0, s>>>(view<double>(f), C, scratch);
    } else {
        if (with_energy)
            energy_solute_kernel<StateView<float>, true><<<nb, DIAG_THREADS, 0, s>>>(view<float>(f), C, scratch);
        else solute_f32_kernel<<<nb, DIAG_THREADS, 0, s>>>(
            (const float*)f.c, (const float*)f.clo, P.cells(), scratch);
    }
    finish_sum2<<<1, DIAG_THREADS, 0, s>>>(scratch, nb, C.dV, out, slot);
    return cudaGetLastError();
}

cudaError_t launch_energy_solute_fields(const HostProblem& P, const void* phi, const void* cs, const void* cl,
                                        int64_t step, int64_t shifts, double* scratch, double* out,
                                        cudaStream_t s) {
    const DiagConsts C = make_diag(P, step, shifts);
    const int nb = diag_blocks(P.cells());
    if (P.precision == 1)
        energy_solute_kernel<FieldView<double>, true><<<nb, DIAG_THREADS, 0, s>>>(
            FieldView<double>{(const double*)phi, (const double*)cs, (const double*)cl}, C, scratch);
    else
        energy_solute_kernel<FieldView<float>, true><<<nb, DIAG_THREADS, 0, s>>>(
            FieldView<float>{(const float*)phi, (const float*)cs, (const float*)cl}, C, scratch);
    finish_sum2<<<1, DIAG_THREADS, 0, s>>>(scratch, nb, C.dV, out, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_front(const HostProblem& P, const Fields& f, double* scratch, double* out,
                         cudaStream_t s) {
    const DiagConsts C = make_diag(P, 0, 0);
    const int nb = diag_blocks(P.cells() / P.n[0]);   // one thread per x row
    if (P.precision == 1)
        front_kernel<double><<<nb, DIAG_THREADS, 0, s>>>(view<double>(f), C, scratch);
    else
        front_kernel<float><<<nb, DIAG_THREADS, 0, s>>>(view<float>(f), C, scratch);
    finish_max2<<<1, DIAG_THREADS, 0, s>>>(scratch, nb, out);
    return cudaGetLastError();
}

static double p_host(const HostProblem& P, double f) {
    const double g = f * (1.0 - f);
    const double h = (P.interp == 1) ? f * f * (3.0 - 2.0 * f) : f * f * f * (6.0 * f * f - 15.0 * f + 10.0);
    return h + P.a * (f - 0.5) * g * g;
}

cudaError_t launch_shift(const HostProblem& P, const Fields& in, const Fields& out, cudaStream_t s) {
    const int n = (int)P.n[0];
    const int blocks = (n + 255) / 256;
    const double p = p_host(P, P.dir_phi);
    const double fc = p * P.dir_cs + (1.0 - p) * P.dir_cl, fd = P.dir_cs - P.dir_cl;
    if (P.precision == 1)
        shift_kernel<double><<<blocks, 256, 0, s>>>(view<double>(in), nullptr, (double*)out.phi,
                                                    (double*)out.c, (double*)out.d, nullptr, nullptr, n,
                                                    P.dir_phi, fc, fd);
    else
        shift_kernel<float><<<blocks, 256, 0, s>>>(view<float>(in), (const float*)in.plo, (float*)out.phi,
                                                   (float*)out.c, (float*)out.d, (float*)out.clo,
                                                   (float*)out.plo, n, P.dir_phi, fc, fd);
    return cudaGetLastError();
}

cudaError_t launch_to_state(const HostProblem& P, const void* phi, const void* cs, const void* cl,
                            const Fields& out, cudaStream_t s) {
    const DiagConsts C = make_diag(P, 0, 0);
    const long long n = P.cells();
    if (P.precision == 1)
        to_state_kernel<double><<<diag_grid(), DIAG_THREADS, 0, s>>>(
            (const double*)phi, (const double*)cs, (const double*)cl, n, C, (double*)out.phi,
            (double*)out.c, (double*)out.d, nullptr);
    else
        to_state_f32((const float*)phi, (const float*)cs, (const float*)cl, n, C, (float*)out.phi,
                     (float*)out.c, (float*)out.d, (float*)out.clo, (float*)out.plo, diag_grid(), s);
    return cudaGetLastError();
}

cudaError_t launch_to_state_range(const HostProblem& P, const void* phi, const void* cs, const void* cl,
                                  const Fields& out, long long first, long long count, int blocks,
                                  cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const DiagConsts C = make_diag(P, 0, 0);
    const int nb = blocks > 0 ? blocks : diag_grid();
    if (P.precision == 1) {
        auto at = [&](const void* p) { return static_cast<const double*>(p) + first; };
        auto to = [&](void* p) { return static_cast<double*>(p) + first; };
        to_state_kernel<double><<<nb, DIAG_THREADS, 0, s>>>(at(phi), at(cs), at(cl), count, C, to(out.phi),
                                                            to(out.c), to(out.d), nullptr);
    } else {
        auto at = [&](const void* p) { return static_cast<const float*>(p) + first; };
        auto to = [&](void* p) { return p ? static_cast<float*>(p) + first : nullptr; };
        to_state_f32(at(phi), at(cs), at(cl), count, C, to(out.phi), to(out.c), to(out.d), to(out.clo),
                     to(out.plo), nb, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_from_state(const HostProblem& P, const Fields& in, void* phi, void* cs, void* cl,
                              cudaStream_t s, int blocks) {
    const DiagConsts C = make_diag(P, 0, 0);
    const long long n = P.cells();
    const int nb = blocks > 0 ? blocks : diag_grid();
    if (P.precision == 1) {
        from_state_kernel<double><<<nb, DIAG_THREADS, 0, s>>>(
            view<double>(in), n, C, (double*)phi, (double*)cs, (double*)cl);
        return cudaGetLastError();
    }
    if (in.clo == nullptr) {   // no low word of c (not a state of this library's FP32 handles)
        from_state_kernel<float><<<nb, DIAG_THREADS, 0, s>>>(
            view<float>(in), n, C, (float*)phi, (float*)cs, (float*)cl);
        return cudaGetLastError();
    }
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const float *f = (const float*)in.phi, *c = (const float*)in.c, *lo = (const float*)in.clo,
                *d = (const float*)in.d;
    long long n4 = 0;
    if (al(f) && al(c) && al(lo) && al(d) && al(phi) && al(cs) && al(cl)) {
        n4 = n / 4;
        if (n4 > 0)
            from_state_f32x4_kernel<<<nb, DIAG_THREADS, 0, s>>>(
                (const float4*)f, (const float4*)c, (const float4*)lo, (const float4*)d, n4, C, (float4*)phi,
                (float4*)cs, (float4*)cl);
    }
    const long long o = 4 * n4;
    if (o < n)
        from_state_f32_kernel<<<nb, DIAG_THREADS, 0, s>>>(f + o, c + o, lo + o, d + o, n - o, C,
                                                                   (float*)phi + o, (float*)cs + o,
                                                                   (float*)cl + o);
    return cudaGetLastError();
}

}  // namespace pf
