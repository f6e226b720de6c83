// pf_noalloc.cu -- pf_energy_solute_noalloc: the FP64 free-energy and
// total-solute reduction of pf_energy / pf_solute_total for callers that
// cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc -- a process whose device
// memory is entirely reserved by another allocator (a framework's caching
// allocator, a fixed arena), monitoring or real-time paths that must not block
// or fail on an allocation, and callers without a pf_handle (creating one
// allocates).  The caller passes device pointers to the fields and to the two
// output doubles; the block partials of the reduction live in a file-scope
// device array instead of a cudaMalloc'd buffer.
//
// The scratch array is shared by every call in the process (and stays resident
// on every GPU that loads the library until exit).  Each call overwrites all
// the partials it later reads, so nothing has to be cleared between calls, but
// two calls whose kernels overlap on the GPU (different streams, no ordering)
// race on it and may return wrong results: serialise them.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include "pf.h"
#include "pf_internal.cuh"
#include "pf_kernels.h"

namespace pf {

static constexpr int NOALLOC_THREADS = 256;
static constexpr int NOALLOC_BLOCKS = 1216;                 // 8 per SM on a 152-SM GB300
static constexpr long long NOALLOC_MAX_CELLS = 1LL << 30;    // largest grid accepted

// block partials of the two sums: 2 x 1216 doubles = 19 KiB
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_BLOCKS];

struct NoallocConsts {
    int n[3], bc_lo[3], bc_hi[3], dim, lap, interp;
    double dir_phi, dx, H, sigma, k_e, a, theta0, G_theta, dV;
};

__device__ __forceinline__ double na_p(const NoallocConsts& C, double f) {
    const double g = f * (1.0 - f);
    const double h = (C.interp == 1) ? f * f * (3.0 - 2.0 * f) : f * f * f * (6.0 * f * f - 15.0 * f + 10.0);
    return h + C.a * (f - 0.5) * g * g;
}

template <typename T>
__device__ __forceinline__ double na_phi(const NoallocConsts& C, const T* phi, int i, int j, int k) {
    const int mi = map_coord(i, C.n[0], C.bc_lo[0], C.bc_hi[0]);
    const int mj = (C.dim >= 2) ? map_coord(j, C.n[1], C.bc_lo[1], C.bc_hi[1]) : 0;
    const int mk = (C.dim >= 3) ? map_coord(k, C.n[2], C.bc_lo[2], C.bc_hi[2]) : 0;
    if (mi < 0 || mj < 0 || mk < 0) return C.dir_phi;
    return (double)phi[((long long)mk * C.n[1] + mj) * C.n[0] + mi];
}

__device__ __forceinline__ double na_warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// per block: partial sums of the energy density and of c over a grid-stride
// range of cells, from (phi, c_s, c_l)
template <typename T>
__global__ void __launch_bounds__(NOALLOC_THREADS)
noalloc_partials(const T* __restrict__ phi, const T* __restrict__ cs, const T* __restrict__ cl,
                 NoallocConsts C, double* __restrict__ part) {
    const long long N = (long long)C.n[0] * C.n[1] * C.n[2];
    double eF = 0.0, eS = 0.0;
    const double one_m_ke = 1.0 - C.k_e, log_ke = log(C.k_e);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % C.n[0]);
        const int j = (int)((c / C.n[0]) % C.n[1]);
        const int k = (int)(c / ((long long)C.n[0] * C.n[1]));
        const double f = (double)phi[c], s = (double)cs[c], l = (double)cl[c];
        const double p = na_p(C, f);
        eS += p * s + (1.0 - p) * l;
        const double theta = C.theta0 - C.G_theta * (((double)i + 0.5) * C.dx);
        const double fs = -one_m_ke * theta + s * (log(s) - log_ke - 1.0);
        const double fl = l * (log(l) - 1.0);
        double gs = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int nz = (dx != 0) + (dy != 0) + (dz != 0);
                    if (nz == 0) continue;
                    double w = 0.0;
                    if (C.lap == 3) w = (dy == 0 && dz == 0) ? 1.0 : 0.0;
                    else if (C.lap == 5) w = (dz == 0 && nz == 1) ? 1.0 : 0.0;
                    else if (C.lap == 9) w = (dz != 0) ? 0.0 : (nz == 1 ? 2.0 / 3.0 : 1.0 / 6.0);
                    else if (C.lap == 7) w = (nz == 1) ? 1.0 : 0.0;
                    else w = (nz == 1) ? 1.0 / 3.0 : (nz == 2 ? 1.0 / 6.0 : 0.0);
                    if (w == 0.0) continue;
                    const double dphi = na_phi(C, phi, i + dx, j + dy, k + dz) - f;
                    gs += w * dphi * dphi;
                }
        eF += C.H * f * f * (1.0 - f) * (1.0 - f) + p * fs + (1.0 - p) * fl +
              0.5 * C.sigma * 0.5 * gs / (C.dx * C.dx);
    }
    __shared__ double sa[NOALLOC_THREADS / 32], sb[NOALLOC_THREADS / 32];
    eF = na_warp_sum(eF);
    eS = na_warp_sum(eS);
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = eF;
        sb[threadIdx.x >> 5] = eS;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < NOALLOC_THREADS / 32; ++w) {
            a += sa[w];
            b += sb[w];
        }
        part[blockIdx.x] = a;
        part[NOALLOC_BLOCKS + blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(NOALLOC_THREADS)
noalloc_finish(const double* __restrict__ part, double scale, double* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < NOALLOC_BLOCKS; i += blockDim.x) {
        a += part[i];
        b += part[NOALLOC_BLOCKS + i];
    }
    __shared__ double sa[NOALLOC_THREADS / 32], sb[NOALLOC_THREADS / 32];
    a = na_warp_sum(a);
    b = na_warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < NOALLOC_THREADS / 32; ++w) {
            x += sa[w];
            y += sb[w];
        }
        out[0] = x * scale;
        out[1] = y * scale;
    }
}

// device address of the scratch array, looked up once per device (the array's
// name in host code is only a host-side stand-in)
static double* scratch_address(int dev, cudaError_t* err) {
    static std::mutex mu;
    static double* addr[64] = {nullptr};
    *err = cudaSuccess;
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        addr[dev] = static_cast<double*>(p);
    }
    return addr[dev];
}

}  // namespace pf

extern "C" int pf_energy_solute_noalloc(const pf_grid* grid, const pf_bc* bc, const pf_params* params,
                                        int64_t step, int64_t shifts, const void* phi, const void* cs,
                                        const void* cl, double* out, void* stream) {
    using namespace pf;
    if (!grid || !bc || !params || !phi || !cs || !cl || !out) {
        set_create_error("pf_energy_solute_noalloc: null argument");
        return PF_EINVAL;
    }
    if (grid->dim < 1 || grid->dim > 3 || !(grid->dx > 0) || !(params->k_e > 0 && params->k_e < 1) ||
        (params->precision != PF_FP32 && params->precision != PF_FP64)) {
        set_create_error("pf_energy_solute_noalloc: invalid grid or parameters");
        return PF_EINVAL;
    }
    long long cells = 1;
    for (int a = 0; a < 3; ++a) {
        const int64_t n = (a < grid->dim) ? grid->n[a] : 1;
        if (n < 1 || (a >= grid->dim && grid->n[a] != 1) || (a < grid->dim && n < 3)) {
            set_create_error("pf_energy_solute_noalloc: invalid grid size");
            return PF_EINVAL;
        }
        if (n > NOALLOC_MAX_CELLS || cells > NOALLOC_MAX_CELLS / n) {
            set_create_error("pf_energy_solute_noalloc: grid exceeds the 2^30-cell maximum");
            return PF_EINVAL;
        }
        cells *= n;
    }
    const int L = params->lap_stencil;
    if ((grid->dim == 1 && L != 3) || (grid->dim == 2 && L != 5 && L != 9) || (grid->dim == 3 && L != 7 && L != 19)) {
        set_create_error("pf_energy_solute_noalloc: lap_stencil does not match dim");
        return PF_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    double* part = (e == cudaSuccess) ? scratch_address(dev, &e) : nullptr;
    if (e != cudaSuccess || !part) {
        set_create_error(std::string("pf_energy_solute_noalloc: scratch set-up: ") + cudaGetErrorString(e));
        return PF_ECUDA;
    }
    NoallocConsts C;
    for (int a = 0; a < 3; ++a) {
        C.n[a] = (int)((a < grid->dim) ? grid->n[a] : 1);
        C.bc_lo[a] = (a < grid->dim) ? bc->lo[a] : PF_BC_NOFLUX;
        C.bc_hi[a] = (a < grid->dim) ? bc->hi[a] : PF_BC_NOFLUX;
    }
    C.dim = grid->dim;
    C.lap = L;
    C.interp = params->interp;
    C.dir_phi = bc->dir_phi;
    C.dx = grid->dx;
    C.H = params->H;
    C.sigma = params->sigma;
    C.k_e = params->k_e;
    C.a = params->a;
    const double t = (double)step * params->dt;
    C.theta0 = params->theta_ref + params->G_theta * (params->x0 + params->v_pull * t - (double)shifts * grid->dx);
    C.G_theta = params->G_theta;
    C.dV = std::pow(grid->dx, grid->dim);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (params->precision == PF_FP64)
        noalloc_partials<double><<<NOALLOC_BLOCKS, NOALLOC_THREADS, 0, s>>>(
            (const double*)phi, (const double*)cs, (const double*)cl, C, part);
    else
        noalloc_partials<float><<<NOALLOC_BLOCKS, NOALLOC_THREADS, 0, s>>>(
            (const float*)phi, (const float*)cs, (const float*)cl, C, part);
    noalloc_finish<<<1, NOALLOC_THREADS, 0, s>>>(part, C.dV, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_create_error(std::string("pf_energy_solute_noalloc: launch: ") + cudaGetErrorString(e));
        return PF_ECUDA;
    }
    return PF_OK;
}
