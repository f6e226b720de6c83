// pf_batch.cu -- batched 1D pulled fronts in one persistent launch.
//
// Each CTA owns one 1D directional-solidification instance (frozen
// temperature of Eq. ds1, moving window of Sec. "Numerical technique",
// no-flux cold end, fixed hot end) and keeps its whole state in shared memory
// for `nsteps` steps: phi, c = p c_s + (1-p) c_l, d = c_s - c_l, the diffusion
// potentials and the phase-field rate.  Global memory is touched only at the
// start and the end of a launch.  The discrete step is the one of the other
// kernels (Eq. phasefield_nonvar with the re-derived driving force at cells;
// the brackets of Eqs. cs_nonvar / cl_nonvar at faces; forward Euler on phi, c,
// d).  Every `check_every` steps the CTA evaluates k_v = c_inf / c_max (Sec.
// "Effect of parameter A on velocity-dependent partition coefficient") and
// marks the instance converged once |dk_v/dt| stays below a tolerance over a
// window of at least `window` time units; converged instances return at once in
// later launches.  Instances are grouped by the block size an autotuner picks
// for their length; the groups run concurrently on forked streams and the whole
// chunk of launches is captured in a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>
#include "pf.h"
#include "pf_dual.cuh"
#include "pf_internal.cuh"
#include "pf_kernels.h"

namespace pf {

constexpr int BATCH_J = 8;   // cells per thread at most

// per-instance persistent state (device)
struct BatchState {
    long long off;      // offset of the instance's cells in the packed field arrays
    int n;              // cells
    int converged;      // 0 running, 1 converged, 2 stopped: the state became non-finite
    long long step, shifts;
    double k_prev, t_prev, k_last, dkdt_last;
};

template <typename T>
struct BatchArgs {
    T* phi;             // packed fields
    T* c;
    T* d;
    BatchState* st;
    const int* ids;     // instances of this launch group
    const double* v;    // per-instance pulling velocity
    const double* dt;   // per-instance time step
    int count;
    int nsteps;
    int check_every;
    double tol, window, min_travel;
    Consts<T> C;        // shared model parameters (dt unused; per instance)
    double theta_ref, G_theta, x0, c_inf;
    T gphi, gcs, gcl, gmus, gmul;   // Dirichlet (hot end) ghost
    T fc, fd;                       // fresh-layer state of the moving window
    int hot_noflux;                 // 1: mirror ghost and zero flux at the hot end too
    long long energy_every;         // record F_h every this many steps (0: never)
    int energy_slots;               // records per instance in `energy`
    double* energy;                 // [instance][slot] F_h records (device)
    double dir_phi;                 // hot-end ghost phi, for the gradient energy
    T* rec;                         // if set: every step's state and intermediates,
                                    // [instance block of 6 rec_steps n][step][phi|c|d|mu_s|mu_l|phidot][n]
    long long rec_steps;
};

template <typename T>
__device__ __forceinline__ T frcp_b(T x) { return T(1) / x; }

// 1D face (L, R): normal differences only
template <typename T>
__device__ __forceinline__ void face1(const Consts<T>& C, T fL, T fR, T csL, T csR, T clL, T clR,
                                      T pdL, T pdR, T nphi, T nY, T nS, T nL, T& Fc, T& Fd) {
    const T f = T(0.5) * (fL + fR);
    const T cs = T(0.5) * (csL + csR), cl = T(0.5) * (clL + clR);
    const T d = cs - cl;
    const T pdot = T(0.5) * (pdL + pdR);
    const T p = p_of(C, f);
    const T omp = T(1) - p;
    const T Ms = Ms_of(C, cs), Ml = Ml_of(C, cl);
    const T bMl = C.b * Ml;
    const T iMbar = frcp_b(Ms * omp + bMl * p);
    const T gt2d = C.delta2;
    const T r = frcp_b(nphi * nphi + gt2d);
    const T Ts = Ms * nS * gt2d;
    const T Tl = Ml * nL * gt2d;
    const T at = C.one_m_A * d * pdot * nphi;
    const T q = Ms * Ml * (C.b * p + omp) * iMbar;
    const T afn = (Ms - bMl) * p * omp * iMbar;
    Fc = r * (q * nphi * nphi * nY + p * Ts + omp * Tl + at * afn);
    Fd = r * (Ts - Tl + at);
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT)
batch_kernel(BatchArgs<T> a) {
    const int inst = a.ids[blockIdx.x];
    BatchState& S = a.st[inst];
    if (S.converged) return;
    const int n = S.n;
    const Consts<T>& C = a.C;
    extern __shared__ __align__(16) unsigned char smem[];
    T* sPhi = reinterpret_cast<T*>(smem);          // n
    T* sC = sPhi + n;                               // n
    T* sD = sC + n;                                 // n
    T* sMs = sD + n;                                // n: mu_s
    T* sMl = sMs + n;                               // n: mu_l
    T* sPd = sMl + n;                               // n: phase-field rate
    __shared__ double red[NT / 32];
    __shared__ int s_done;

    const int tid = threadIdx.x;
    const long long off = S.off;
    for (int i = tid; i < n; i += NT) {
        sPhi[i] = a.phi[off + i];
        sC[i] = a.c[off + i];
        sD[i] = a.d[off + i];
    }
    long long step = S.step, shifts = S.shifts;
    double k_prev = S.k_prev, t_prev = S.t_prev, k_last = S.k_last, dkdt_last = S.dkdt_last;
    int converged = 0;
    const double v = a.v[inst];
    const T dt = T(a.dt[inst]);
    const T dtdx = dt * C.inv_dx;
    if (tid == 0) s_done = 0;
    __syncthreads();

    auto cs_cl = [&](int i, T& p, T& cs, T& cl) {
        p = p_of(C, sPhi[i]);
        cs = sC[i] + (T(1) - p) * sD[i];
        cl = sC[i] - p * sD[i];
    };

    for (int it = 0; it < a.nsteps; ++it) {
        const double t = (double)step * a.dt[inst];
        const T theta0 = T(a.theta_ref + a.G_theta * (a.x0 + v * t - (double)shifts * (double)C.dx));
        // for a reverse sweep: the pre-step state, then mu_s, mu_l, phidot below
        T* const rec = a.rec != nullptr ? a.rec + 6 * a.rec_steps * off + (long long)it * 6 * n : nullptr;
        if (rec != nullptr) {
            for (int i = tid; i < n; i += NT) {
                rec[i] = sPhi[i];
                rec[n + i] = sC[i];
                rec[2 * n + i] = sD[i];
            }
        }
        // P1: diffusion potentials
        for (int i = tid; i < n; i += NT) {
            T p, cs, cl;
            cs_cl(i, p, cs, cl);
            sMs[i] = flog(cs) - C.log_ke;
            sMl[i] = flog(cl);
            if (rec != nullptr) {
                rec[3 * n + i] = sMs[i];
                rec[4 * n + i] = sMl[i];
            }
        }
        __syncthreads();
        // P2: phase-field rate (cold end: mirror ghost; hot end: Dirichlet or
        // mirror ghost)
        for (int i = tid; i < n; i += NT) {
            const int im = (i == 0) ? 0 : i - 1;
            const bool last = i == n - 1, mirror_hot = last && a.hot_noflux;
            const int ip = last ? i : i + 1;
            const T fc = sPhi[i];
            const T fW = sPhi[im];
            const T fE = (last && !mirror_hot) ? a.gphi : sPhi[ip];
            const T mW_s = sMs[im], mW_l = sMl[im];
            const T mE_s = (last && !mirror_hot) ? a.gmus : sMs[ip];
            const T mE_l = (last && !mirror_hot) ? a.gmul : sMl[ip];
            T p, cs, cl;
            cs_cl(i, p, cs, cl);
            const T mus = sMs[i], mul = sMl[i];
            const T dp = dp_of(C, fc);
            const T lap = (fW - T(2) * fc + fE) * C.inv_dx2;
            const T gp = (fE - fW) * C.inv_2dx;
            const T gs = (mE_s - mW_s) * C.inv_2dx;
            const T gl = (mE_l - mW_l) * C.inv_2dx;
            const T Ms = Ms_of(C, cs), Ml = Ml_of(C, cl);
            const T bMl = C.b * Ml;
            const T Msq = Ms * (T(1) - p);
            const T iMbar = frcp_b(Msq + bMl * p);
            const T d = cs - cl;
            const T rr = frcp_b(gp * gp + C.delta2);
            const T pq = p * (T(1) - p);
            const T Kc = C.inv_Mphi + C.one_m_A * C.one_m_A * d * d * C.b * pq * rr * iMbar /
                                          (C.b * p + T(1) - p);
            const T theta = theta0 - C.G_theta * ((T(i) + T(0.5)) * C.dx);
            const T dmu = mus - mul;
            const T Dd = (Msq * (T(1) - C.A * (T(1) - p)) + C.A * bMl * p * p) * iMbar;
            const T dG = cs * dmu - d - C.one_m_ke * theta - Dd * d * dmu;
            const T dfdw = T(2) * fc * (T(1) - fc) * (T(1) - T(2) * fc);
            const T R = C.sigma * lap - C.H * dfdw - dG * dp +
                        C.one_m_A * d * pq * iMbar * (Ms * gs - bMl * gl) * gp * rr;
            sPd[i] = R / Kc;
            if (rec != nullptr) rec[5 * n + i] = sPd[i];
        }
        __syncthreads();
        // P3: faces of each owned cell and the new state (kept in registers)
        T nphi[BATCH_J], nc[BATCH_J], nd[BATCH_J];
#pragma unroll
        for (int j = 0; j < BATCH_J; ++j) {
            const int i = tid + j * NT;
            if (i >= n) break;
            T pL, csL, clL, pR, csR, clR, p0, cs0, cl0;
            cs_cl(i, p0, cs0, cl0);
            const T f0 = sPhi[i], ms0 = sMs[i], ml0 = sMl[i], pd0 = sPd[i];
            const T Y0 = ml0 + p0 * (ms0 - ml0);
            T FcL = T(0), FdL = T(0), FcR, FdR;
            if (i > 0) {   // face (i-1, i); the face at the cold end is no-flux
                cs_cl(i - 1, pL, csL, clL);
                const T fL = sPhi[i - 1], msL = sMs[i - 1], mlL = sMl[i - 1];
                const T YL = mlL + pL * (msL - mlL);
                face1(C, fL, f0, csL, cs0, clL, cl0, sPd[i - 1], pd0, (f0 - fL) * C.inv_dx,
                      (Y0 - YL) * C.inv_dx, (ms0 - msL) * C.inv_dx, (ml0 - mlL) * C.inv_dx, FcL, FdL);
            }
            if (i < n - 1) {
                cs_cl(i + 1, pR, csR, clR);
                const T fR = sPhi[i + 1], msR = sMs[i + 1], mlR = sMl[i + 1];
                const T YR = mlR + pR * (msR - mlR);
                face1(C, f0, fR, cs0, csR, cl0, clR, pd0, sPd[i + 1], (fR - f0) * C.inv_dx,
                      (YR - Y0) * C.inv_dx, (msR - ms0) * C.inv_dx, (mlR - ml0) * C.inv_dx, FcR, FdR);
            } else if (a.hot_noflux) {   // closed hot end: no flux through the last face
                FcR = T(0);
                FdR = T(0);
            } else {       // face to the fixed hot-end ghost (phase-field rate 0)
                const T gp = p_of(C, a.gphi);
                const T YR = a.gmul + gp * (a.gmus - a.gmul);
                face1(C, f0, a.gphi, cs0, a.gcs, cl0, a.gcl, pd0, T(0), (a.gphi - f0) * C.inv_dx,
                      (YR - Y0) * C.inv_dx, (a.gmus - ms0) * C.inv_dx, (a.gmul - ml0) * C.inv_dx, FcR, FdR);
            }
            nphi[j] = f0 + dt * pd0;
            nc[j] = sC[i] + dtdx * (FcR - FcL);
            nd[j] = sD[i] + dtdx * (FdR - FdL);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < BATCH_J; ++j) {
            const int i = tid + j * NT;
            if (i >= n) break;
            sPhi[i] = nphi[j];
            sC[i] = nc[j];
            sD[i] = nd[j];
        }
        step += 1;
        // moving window: drop the cold-end cell, append the fresh hot-end state
        const double tn = (double)step * a.dt[inst];
        while (v * tn >= (double)(shifts + 1) * (double)C.dx) {
            __syncthreads();
#pragma unroll
            for (int j = 0; j < BATCH_J; ++j) {
                const int i = tid + j * NT;
                if (i >= n) break;
                if (i < n - 1) {
                    nphi[j] = sPhi[i + 1]; nc[j] = sC[i + 1]; nd[j] = sD[i + 1];
                } else {
                    nphi[j] = a.gphi; nc[j] = a.fc; nd[j] = a.fd;
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < BATCH_J; ++j) {
                const int i = tid + j * NT;
                if (i >= n) break;
                sPhi[i] = nphi[j]; sC[i] = nc[j]; sD[i] = nd[j];
            }
            shifts += 1;
        }
        __syncthreads();
        // F_h of the new state (the discrete free energy of pf_energy), FP64
        if (a.energy_every > 0 && (step % a.energy_every) == 0) {
            const double t = (double)step * a.dt[inst];
            const double th0 = a.theta_ref + a.G_theta * (a.x0 + v * t - (double)shifts * (double)C.dx);
            const double dxd = (double)C.dx, ke = (double)C.one_m_ke;
            double e = 0.0;
            for (int i = tid; i < n; i += NT) {
                const double f = (double)sPhi[i], cc = (double)sC[i], dd = (double)sD[i];
                const double g = f * (1.0 - f);
                const double h = f * f * ((double)C.h2 + f * ((double)C.h3 + f * ((double)C.h4 + f * (double)C.h5)));
                const double p = h + (double)C.a * (f - 0.5) * g * g;
                const double cs = cc + (1.0 - p) * dd, cl = cc - p * dd;
                const double th = th0 - (double)C.G_theta * (((double)i + 0.5) * dxd);
                const double fs = -ke * th + cs * (log(cs) - (double)C.log_ke - 1.0);
                const double fl = cl * (log(cl) - 1.0);
                // gradient energy: each pair of cells once, from its left cell;
                // mirror ghosts add nothing and the pair with a Dirichlet ghost
                // counts half, as in pf_energy
                double gs = 0.0;
                if (i < n - 1) {
                    const double dphi = (double)sPhi[i + 1] - f;
                    gs = dphi * dphi;
                } else if (!a.hot_noflux) {
                    const double dphi = a.dir_phi - f;
                    gs = 0.5 * dphi * dphi;
                }
                e += (double)C.H * g * g + p * fs + (1.0 - p) * fl + 0.5 * (double)C.sigma * gs / (dxd * dxd);
            }
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
            if ((tid & 31) == 0) red[tid >> 5] = e;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int w = 0; w < NT / 32; ++w) tot += red[w];
                const long long slot = step / a.energy_every - 1;
                if (slot < a.energy_slots) a.energy[(long long)inst * a.energy_slots + slot] = tot * dxd;
            }
            __syncthreads();
        }
        // steady-state check on k_v = c_inf / c_max
        if (a.check_every > 0 && (step % a.check_every) == 0) {
            // a maximum that keeps a NaN (fmax would drop it): a state that has
            // stopped being finite must not look steady
            auto nanmax = [](double x, double y) { return (y > x || y != y) ? y : x; };
            double cm = -1e300;
            for (int i = tid; i < n; i += NT) cm = nanmax(cm, (double)sC[i]);
            for (int o = 16; o > 0; o >>= 1) cm = nanmax(cm, __shfl_xor_sync(0xffffffffu, cm, o));
            if ((tid & 31) == 0) red[tid >> 5] = cm;
            __syncthreads();
            if (tid == 0) {
                double m = red[0];
                for (int w = 1; w < NT / 32; ++w) m = nanmax(m, red[w]);
                const double k = a.c_inf / m;
                k_last = k;
                if (!isfinite(m)) {
                    s_done = 2;   // non-finite state: the instance stops, not converged
                } else if (tn - t_prev >= a.window) {
                    dkdt_last = fabs(k - k_prev) / (tn - t_prev);
                    s_done = (t_prev > 0.0 && dkdt_last < a.tol && v * tn >= a.min_travel) ? 1 : 0;
                    k_prev = k;
                    t_prev = tn;
                }
            }
            __syncthreads();
            if (s_done) {
                converged = s_done;
                break;
            }
        }
    }
    for (int i = tid; i < n; i += NT) {
        a.phi[off + i] = sPhi[i];
        a.c[off + i] = sC[i];
        a.d[off + i] = sD[i];
    }
    if (tid == 0) {
        S.step = step;
        S.shifts = shifts;
        S.k_prev = k_prev;
        S.t_prev = t_prev;
        S.k_last = k_last;
        S.dkdt_last = dkdt_last;
        S.converged = converged;
    }
}


// (phi, c_s, c_l) -> (phi, c, d) for packed instances
template <typename T>
__global__ void batch_to_state(const T* __restrict__ cs, const T* __restrict__ cl, T* __restrict__ phi,
                               T* __restrict__ c, T* __restrict__ d, long long n, int interp, double a) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double f = (double)phi[i], s = (double)cs[i], l = (double)cl[i];
        const double g = f * (1.0 - f);
        const double h = (interp == 1) ? f * f * (3.0 - 2.0 * f) : f * f * f * (6.0 * f * f - 15.0 * f + 10.0);
        const double p = h + a * (f - 0.5) * g * g;
        c[i] = (T)(p * s + (1.0 - p) * l);
        d[i] = (T)(s - l);
    }
}

template <typename T>
__global__ void batch_from_state(const T* __restrict__ phi, const T* __restrict__ c, const T* __restrict__ d,
                                 T* __restrict__ cs, T* __restrict__ cl, long long n, int interp, double a) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double f = (double)phi[i], cc = (double)c[i], dd = (double)d[i];
        const double g = f * (1.0 - f);
        const double h = (interp == 1) ? f * f * (3.0 - 2.0 * f) : f * f * f * (6.0 * f * f - 15.0 * f + 10.0);
        const double p = h + a * (f - 0.5) * g * g;
        cs[i] = (T)(cc + (1.0 - p) * dd);
        cl[i] = (T)(cc - p * dd);
    }
}

namespace {

double p_of_host(const pf_params& P, double f) {
    const double g = f * (1.0 - f);
    const double h = (P.interp == 1) ? f * f * (3.0 - 2.0 * f) : f * f * f * (6.0 * f * f - 15.0 * f + 10.0);
    return h + P.a * (f - 0.5) * g * g;
}

int threads_for(int64_t n, int cpt) {
    int nt = 128;
    while (nt < 1024 && (int64_t)nt * cpt < n) nt *= 2;
    return nt;
}

template <typename T>
cudaError_t launch_group(int nt, const BatchArgs<T>& a, size_t smem, cudaStream_t s) {
    switch (nt) {
        case 128: batch_kernel<T, 128><<<a.count, 128, smem, s>>>(a); break;
        case 256: batch_kernel<T, 256><<<a.count, 256, smem, s>>>(a); break;
        case 512: batch_kernel<T, 512><<<a.count, 512, smem, s>>>(a); break;
        default: batch_kernel<T, 1024><<<a.count, 1024, smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

// raise each instantiation's dynamic shared-memory limit to what the device
// allows next to the kernel's static shared memory
template <typename K>
cudaError_t raise_smem(K kern, int optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

template <typename T>
cudaError_t set_smem_limits(size_t* max_dynamic) {
    static DeviceSetup setup;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= DeviceSetup::MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(setup.mu);
    if (!setup.done[dev]) {
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = raise_smem(batch_kernel<T, 128>, optin);
        if (e == cudaSuccess) e = raise_smem(batch_kernel<T, 256>, optin);
        if (e == cudaSuccess) e = raise_smem(batch_kernel<T, 512>, optin);
        if (e == cudaSuccess) e = raise_smem(batch_kernel<T, 1024>, optin);
        setup.value[dev] = (size_t)optin - 1024;   // static part: reduction scratch and flag
        setup.err[dev] = e;
        setup.done[dev] = true;
    }
    *max_dynamic = setup.value[dev];
    return setup.err[dev];
}

struct Group {
    int nt;
    int dir = -1;      // seeded parameter of a tangent run (0 M_phi, 1 A, 2 b), -1 none
    int nmax;
    std::vector<int> ids;
    int* d_ids = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

template <typename T>
struct BatchRun {
    const pf_batch_desc& D;
    cudaStream_t main;
    std::string& err;
    int64_t total = 0;
    std::vector<int64_t> off;
    std::vector<double> dt;
    T *phi = nullptr, *c = nullptr, *d = nullptr;
    BatchState* st = nullptr;
    double *dv = nullptr, *ddt = nullptr;
    std::vector<Group> groups;
    std::vector<int> rep_dir;   // tangent runs: seeded parameter of each instance
    double* energy = nullptr;   // F_h records [instance][slot] (device), or null
    int energy_slots = 0;
    T* rec = nullptr;           // reverse sweeps: per-step state record (not owned)
    long long rec_steps = 0;
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    int64_t launches = 0;

    BatchRun(const pf_batch_desc& d_, cudaStream_t s, std::string& e) : D(d_), main(s), err(e) {}
    ~BatchRun() {
        for (Group& g : groups) {
            if (g.d_ids) cudaFree(g.d_ids);
            if (g.stream) cudaStreamDestroy(g.stream);
            if (g.done) cudaEventDestroy(g.done);
        }
        void* ptrs[] = {phi, c, d, st, dv, ddt, energy};
        for (void* p : ptrs)
            if (p) cudaFree(p);
        if (fork) cudaEventDestroy(fork);
        if (t0) cudaEventDestroy(t0);
        if (t1) cudaEventDestroy(t1);
    }

    BatchArgs<T> args(const Group& g, int nsteps) const {
        BatchArgs<T> a;
        a.phi = phi; a.c = c; a.d = d; a.st = st; a.ids = g.d_ids; a.v = dv; a.dt = ddt;
        a.count = (int)g.ids.size();
        a.nsteps = nsteps;
        a.check_every = (int)D.check_every;
        a.tol = D.tol;
        a.window = D.window;
        a.min_travel = D.min_travel;
        const pf_params& P = D.params;
        Consts<T>& C = a.C;
        C = Consts<T>{};   // every member zero (Dual members by their constructor)
        C.dim = 1; C.interp = P.interp; C.lap = 3; C.mobility = P.mobility_mode;
        C.dx = T(D.dx); C.inv_dx = T(1.0 / D.dx); C.inv_2dx = T(0.5 / D.dx); C.inv_dx2 = T(1.0 / (D.dx * D.dx));
        C.H = T(P.H); C.sigma = T(P.sigma); C.inv_Mphi = T(1.0 / P.M_phi); C.D_s = T(P.D_s); C.D_l = T(P.D_l);
        C.log_ke = T(std::log(P.k_e)); C.one_m_ke = T(1.0 - P.k_e); C.A = T(P.A); C.one_m_A = T(1.0 - P.A);
        C.b = T(P.b); C.a = T(P.a); C.delta2 = T(P.delta * P.delta); C.G_theta = T(P.G_theta);
        set_coefficients(C);
        a.theta_ref = P.theta_ref; a.G_theta = P.G_theta; a.x0 = P.x0; a.c_inf = P.c_inf;
        a.gphi = T(D.bc.dir_phi); a.gcs = T(D.bc.dir_cs); a.gcl = T(D.bc.dir_cl);
        a.gmus = T(std::log(D.bc.dir_cs) - std::log(P.k_e));
        a.gmul = T(std::log(D.bc.dir_cl));
        const double pg = p_of_host(P, D.bc.dir_phi);
        a.fc = T(pg * D.bc.dir_cs + (1.0 - pg) * D.bc.dir_cl);
        a.fd = T(D.bc.dir_cs - D.bc.dir_cl);
        a.hot_noflux = D.bc.hi[0] == PF_BC_NOFLUX;
        a.energy_every = D.energy_every;
        a.energy_slots = energy_slots;
        a.energy = energy;
        a.dir_phi = D.bc.dir_phi;
        a.rec = rec;
        a.rec_steps = rec_steps;
        if constexpr (IsDual<T>::value) {
            // seed d/dtheta = 1 on the parameter of this group
            using VT = decltype(C.A.v);
            if (g.dir == 0) C.inv_Mphi = make_dual<VT>(VT(1.0 / P.M_phi), VT(-1.0 / (P.M_phi * P.M_phi)));
            if (g.dir == 1) {
                C.A = make_dual<VT>(VT(P.A), VT(1));
                C.one_m_A = make_dual<VT>(VT(1.0 - P.A), VT(-1));
            }
            if (g.dir == 2) C.b = make_dual<VT>(VT(P.b), VT(1));
        }
        return a;
    }

    cudaError_t issue(int nsteps) {
        cudaError_t e = cudaEventRecord(fork, main);
        for (Group& g : groups) {
            if (e == cudaSuccess) e = cudaStreamWaitEvent(g.stream, fork, 0);
            if (e == cudaSuccess) e = launch_group<T>(g.nt, args(g, nsteps), (size_t)6 * g.nmax * sizeof(T), g.stream);
            if (e == cudaSuccess) e = cudaEventRecord(g.done, g.stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(main, g.done, 0);
            launches += 1;
        }
        return e;
    }

    cudaError_t make_groups(int cpt) {
        for (Group& g : groups) {
            if (g.d_ids) cudaFree(g.d_ids);
            if (g.stream) cudaStreamDestroy(g.stream);
            if (g.done) cudaEventDestroy(g.done);
        }
        groups.clear();
        std::map<std::pair<int, int>, Group> by;
        for (int i = 0; i < D.n_instances; ++i) {
            const int nt = threads_for(D.n[i], cpt);
            const int dir = rep_dir.empty() ? -1 : rep_dir[i];
            Group& g = by[{nt, dir}];
            g.nt = nt;
            g.dir = dir;
            g.nmax = std::max(g.nmax, (int)D.n[i]);
            g.ids.push_back(i);
        }
        // largest instances first inside a group: the long CTAs start early
        for (auto& kv : by) {
            Group g = kv.second;
            std::sort(g.ids.begin(), g.ids.end(), [&](int x, int y) { return D.n[x] > D.n[y]; });
            cudaError_t e = cudaMalloc(&g.d_ids, g.ids.size() * sizeof(int));
            if (e == cudaSuccess) e = cudaMemcpy(g.d_ids, g.ids.data(), g.ids.size() * sizeof(int), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
            groups.push_back(g);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
};

}  // namespace

// per-instance time step: the given one, or 0.9 of the stable step capped so
// that the window moves at most half a cell per step
static bool batch_time_steps(const pf_batch_desc& D, std::vector<double>& out, std::string& err) {
    pf_grid g1{1, {8, 1, 1}, D.dx};
    double dts = 0;
    pf_stable_dt(&g1, &D.params, &dts);
    out.resize(D.n_instances);
    for (int i = 0; i < D.n_instances; ++i) {
        double dt = (D.dt && D.dt[i] > 0) ? D.dt[i] : 0.9 * dts;
        if (!(D.dt && D.dt[i] > 0) && D.v_pull[i] > 0) dt = std::min(dt, 0.5 * D.dx / D.v_pull[i]);
        if (!(dt > 0) || dt > dts * (1 + 1e-12) || D.v_pull[i] * dt >= D.dx) {
            err = "invalid or unstable time step for instance " + std::to_string(i);
            return false;
        }
        out[i] = dt;
    }
    return true;
}

template <typename T>
static int run_batch_T(const pf_batch_desc& D, pf_batch_result* R, cudaStream_t main, std::string& err) {
    BatchRun<T> B(D, main, err);
    const int N = D.n_instances;
    B.off.resize(N);
    B.dt.resize(N);
    for (int i = 0; i < N; ++i) {
        B.off[i] = B.total;
        B.total += D.n[i];
    }
    if (!batch_time_steps(D, B.dt, err)) return PF_EINVAL;
    const size_t fb = (size_t)B.total * sizeof(T);
    cudaError_t e = cudaMalloc(&B.phi, fb);
    if (e == cudaSuccess) e = cudaMalloc(&B.c, fb);
    if (e == cudaSuccess) e = cudaMalloc(&B.d, fb);
    if (e == cudaSuccess) e = cudaMalloc(&B.st, N * sizeof(BatchState));
    if (e == cudaSuccess) e = cudaMalloc(&B.dv, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&B.ddt, N * sizeof(double));
    if (e == cudaSuccess && D.energy_every > 0) {
        // one record per energy_every steps up to max_steps, NaN where never written
        const int64_t slots = D.max_steps / D.energy_every;
        B.energy_slots = (int)slots;
        e = cudaMalloc(&B.energy, (size_t)N * slots * sizeof(double));
        if (e == cudaSuccess) e = cudaMemsetAsync(B.energy, 0xff, (size_t)N * slots * sizeof(double), main);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = std::string("device allocation failed: ") + cudaGetErrorString(e);
        return PF_ENOMEM;
    }
    T *scs = nullptr, *scl = nullptr;
    e = cudaMalloc(&scs, fb);
    if (e == cudaSuccess) e = cudaMalloc(&scl, fb);
    if (e != cudaSuccess) {
        if (scs) cudaFree(scs);
        cudaGetLastError();
        err = "device allocation failed";
        return PF_ENOMEM;
    }
    std::vector<BatchState> hs(N);
    for (int i = 0; i < N; ++i) {
        hs[i] = BatchState{B.off[i], (int)D.n[i], 0, 0, 0, 0.0, 0.0, 0.0, 0.0};
    }
    e = cudaMemcpyAsync(B.phi, D.phi0, fb, cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scs, D.cs0, fb, cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scl, D.cl0, fb, cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.st, hs.data(), N * sizeof(BatchState), cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.dv, D.v_pull, N * sizeof(double), cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.ddt, B.dt.data(), N * sizeof(double), cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) {
        batch_to_state<T><<<1216, 256, 0, main>>>(scs, scl, B.phi, B.c, B.d, B.total, D.params.interp, D.params.a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(main);
    cudaFree(scs);
    cudaFree(scl);
    size_t max_dyn = 0;
    if (e == cudaSuccess) e = set_smem_limits<T>(&max_dyn);
    if (e == cudaSuccess) {
        int64_t nbig = 0;
        for (int i = 0; i < N; ++i) nbig = std::max(nbig, (int64_t)D.n[i]);
        if ((size_t)6 * nbig * sizeof(T) > max_dyn) {
            err = "longest instance does not fit in shared memory";
            return PF_EINVAL;
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&B.t0);
    if (e == cudaSuccess) e = cudaEventCreate(&B.t1);
    if (e != cudaSuccess) {
        err = std::string("batch set-up: ") + cudaGetErrorString(e);
        return PF_ECUDA;
    }

    // autotune the cells per thread: time a short probe of every candidate on a
    // scratch copy of the initial state
    int cpt = D.cells_per_thread;
    if (cpt == 0) {
        T *bp = nullptr, *bc = nullptr, *bd = nullptr;
        e = cudaMalloc(&bp, fb);
        if (e == cudaSuccess) e = cudaMalloc(&bc, fb);
        if (e == cudaSuccess) e = cudaMalloc(&bd, fb);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bp, B.phi, fb, cudaMemcpyDeviceToDevice, main);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bc, B.c, fb, cudaMemcpyDeviceToDevice, main);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bd, B.d, fb, cudaMemcpyDeviceToDevice, main);
        float best = 1e30f;
        const int probe = 32;
        for (int cand : {1, 2, 4, 8}) {
            if (e != cudaSuccess) break;
            bool ok = true;
            for (int i = 0; i < N; ++i)
                if (D.n[i] > (int64_t)1024 * cand) ok = false;
            if (!ok) continue;
            e = B.make_groups(cand);
            if (e == cudaSuccess) e = cudaEventRecord(B.t0, main);
            if (e == cudaSuccess) e = B.issue(probe);
            if (e == cudaSuccess) e = cudaEventRecord(B.t1, main);
            if (e == cudaSuccess) e = cudaEventSynchronize(B.t1);
            float ms = 0;
            if (e == cudaSuccess) cudaEventElapsedTime(&ms, B.t0, B.t1);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                cpt = cand;
            }
            // restore the state the probe advanced
            if (e == cudaSuccess) e = cudaMemcpyAsync(B.phi, bp, fb, cudaMemcpyDeviceToDevice, main);
            if (e == cudaSuccess) e = cudaMemcpyAsync(B.c, bc, fb, cudaMemcpyDeviceToDevice, main);
            if (e == cudaSuccess) e = cudaMemcpyAsync(B.d, bd, fb, cudaMemcpyDeviceToDevice, main);
            if (e == cudaSuccess) e = cudaMemcpyAsync(B.st, hs.data(), N * sizeof(BatchState), cudaMemcpyHostToDevice, main);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(main);
        if (bp) cudaFree(bp);
        if (bc) cudaFree(bc);
        if (bd) cudaFree(bd);
        if (e != cudaSuccess) {
            err = std::string("batch autotune: ") + cudaGetErrorString(e);
            return PF_ECUDA;
        }
        B.launches = 0;
    }
    e = B.make_groups(cpt);
    if (e != cudaSuccess) {
        err = std::string("batch groups: ") + cudaGetErrorString(e);
        return PF_ECUDA;
    }

    // capture a chunk of launches as a CUDA graph and replay it
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    e = cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal);
    for (int l = 0; l < D.launches_per_graph && e == cudaSuccess; ++l) e = B.issue((int)D.steps_per_launch);
    cudaError_t e2 = cudaStreamEndCapture(main, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        err = std::string("batch graph: ") + cudaGetErrorString(e);
        return PF_ECUDA;
    }
    const int64_t per_replay = D.steps_per_launch * D.launches_per_graph;
    B.launches = 0;
    float total_ms = 0;
    int64_t done_steps = 0;
    for (;;) {
        // whole graph replays, then the remainder of max_steps launched directly,
        // so that no instance takes more than max_steps steps
        const int64_t left = D.max_steps - done_steps;
        const bool whole = left >= per_replay;
        e = cudaEventRecord(B.t0, main);
        if (whole) {
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, main);
        } else {
            for (int64_t r = left; r > 0 && e == cudaSuccess; r -= D.steps_per_launch)
                e = B.issue((int)std::min<int64_t>(r, D.steps_per_launch));
        }
        if (e == cudaSuccess) e = cudaEventRecord(B.t1, main);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), B.st, N * sizeof(BatchState), cudaMemcpyDeviceToHost, main);
        if (e == cudaSuccess) e = cudaStreamSynchronize(main);
        if (e != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, B.t0, B.t1);
        total_ms += ms;
        if (whole) B.launches += (int64_t)D.launches_per_graph * (int64_t)B.groups.size();
        done_steps += whole ? per_replay : left;
        bool all = true;
        for (int i = 0; i < N; ++i)
            if (!hs[i].converged) all = false;
        if (all || done_steps >= D.max_steps) break;
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        err = std::string("batch run: ") + cudaGetErrorString(e);
        return PF_ECUDA;
    }
    for (int i = 0; i < N; ++i) {
        if (R->k_v) R->k_v[i] = hs[i].k_last;
        if (R->dkdt) R->dkdt[i] = hs[i].dkdt_last;
        if (R->t) R->t[i] = (double)hs[i].step * B.dt[i];
        if (R->steps) R->steps[i] = hs[i].step;
        if (R->converged) R->converged[i] = hs[i].converged == 1 ? 1 : 0;
    }
    R->cells_per_thread = cpt;
    R->launches = B.launches;
    R->gpu_ms = total_ms;
    if (R->energy && B.energy) {
        e = cudaMemcpyAsync(R->energy, B.energy, (size_t)N * B.energy_slots * sizeof(double),
                            cudaMemcpyDeviceToHost, main);
        if (e == cudaSuccess) e = cudaStreamSynchronize(main);
        if (e != cudaSuccess) {
            err = std::string("batch energy records: ") + cudaGetErrorString(e);
            return PF_ECUDA;
        }
    }
    if (R->phi && R->cs && R->cl) {
        T *ocs = nullptr, *ocl = nullptr;
        e = cudaMalloc(&ocs, fb);
        if (e == cudaSuccess) e = cudaMalloc(&ocl, fb);
        if (e == cudaSuccess) {
            batch_from_state<T><<<1216, 256, 0, main>>>(B.phi, B.c, B.d, ocs, ocl, B.total, D.params.interp, D.params.a);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(R->phi, B.phi, fb, cudaMemcpyDeviceToHost, main);
        if (e == cudaSuccess) e = cudaMemcpyAsync(R->cs, ocs, fb, cudaMemcpyDeviceToHost, main);
        if (e == cudaSuccess) e = cudaMemcpyAsync(R->cl, ocl, fb, cudaMemcpyDeviceToHost, main);
        if (e == cudaSuccess) e = cudaStreamSynchronize(main);
        if (ocs) cudaFree(ocs);
        if (ocl) cudaFree(ocl);
        if (e != cudaSuccess) {
            err = std::string("batch fields: ") + cudaGetErrorString(e);
            return PF_ECUDA;
        }
    }
    return PF_OK;
}

// Runs on a private non-blocking stream forked from the caller's (which may be
// the legacy default stream, not capturable) and joined back at the end.
template <typename T>
static int run_batch_forked(const pf_batch_desc& D, pf_batch_result* R, cudaStream_t caller, std::string& err) {
    cudaStream_t work = nullptr;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&work, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(work, ev, 0);
    int rc = PF_ECUDA;
    if (e == cudaSuccess) {
        rc = run_batch_T<T>(D, R, work, err);
        cudaError_t e2 = cudaEventRecord(ev, work);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(caller, ev, 0);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(work);
        if (rc == PF_OK && e2 != cudaSuccess) {
            err = std::string("batch join: ") + cudaGetErrorString(e2);
            rc = PF_ECUDA;
        }
    } else {
        err = std::string("batch stream: ") + cudaGetErrorString(e);
    }
    if (ev) cudaEventDestroy(ev);
    if (work) cudaStreamDestroy(work);
    return rc;
}

int run_batch(const pf_batch_desc* D, pf_batch_result* R, void* stream, std::string& err) {
    if (!D || !R) { err = "null argument"; return PF_EINVAL; }
    const pf_params& P = D->params;
    const int64_t nmax = (P.precision == PF_FP64) ? 4096 : 8192;
    if (D->n_instances <= 0 || !D->n || !D->v_pull || !D->phi0 || !D->cs0 || !D->cl0) {
        err = "empty batch or null array";
        return PF_EINVAL;
    }
    for (int i = 0; i < D->n_instances; ++i) {
        if (D->n[i] < 8 || D->n[i] > nmax) { err = "instance length outside 8.." + std::to_string(nmax); return PF_EINVAL; }
        if (!(D->v_pull[i] >= 0) || !std::isfinite(D->v_pull[i])) { err = "negative or non-finite velocity"; return PF_EINVAL; }
    }
    if (!(D->dx > 0) || !(P.k_e > 0 && P.k_e < 1) || !(P.b > 0) || !(P.M_phi > 0) || !(P.H > 0) ||
        !(P.sigma > 0) || !(P.D_s > 0) || !(P.D_l > 0) || !(P.c_inf > 0)) {
        err = "invalid model parameters";
        return PF_EINVAL;
    }
    if (P.precision != PF_FP32 && P.precision != PF_FP64) { err = "precision must be PF_FP32 or PF_FP64"; return PF_EINVAL; }
    if (D->bc.lo[0] != PF_BC_NOFLUX || (D->bc.hi[0] != PF_BC_DIRICHLET && D->bc.hi[0] != PF_BC_NOFLUX)) {
        err = "batch instances need a no-flux cold end and a Dirichlet or no-flux hot end";
        return PF_EINVAL;
    }
    if (D->energy_every < 0 || (D->energy_every > 0 && D->max_steps / D->energy_every > (int64_t)1 << 26)) {
        err = "energy_every must be 0 or leave at most 2^26 records per instance";
        return PF_EINVAL;
    }
    if (D->bc.hi[0] == PF_BC_NOFLUX) {
        for (int i = 0; i < D->n_instances; ++i)
            if (D->v_pull[i] != 0.0) { err = "a moving window needs the Dirichlet hot end"; return PF_EINVAL; }
    }
    if (!(D->bc.dir_cs > 0) || !(D->bc.dir_cl > 0)) { err = "Dirichlet concentrations must be positive"; return PF_EINVAL; }
    if (D->steps_per_launch <= 0 || D->launches_per_graph <= 0 || D->check_every <= 0 || D->max_steps <= 0 ||
        D->steps_per_launch > (1 << 30)) {
        err = "steps_per_launch, launches_per_graph, check_every and max_steps must be positive";
        return PF_EINVAL;
    }
    const int cpt = D->cells_per_thread;
    if (cpt != 0 && cpt != 1 && cpt != 2 && cpt != 4 && cpt != 8) { err = "cells_per_thread must be 0, 1, 2, 4 or 8"; return PF_EINVAL; }
    if (cpt != 0)
        for (int i = 0; i < D->n_instances; ++i)
            if (D->n[i] > (int64_t)1024 * cpt) { err = "cells_per_thread too small for the longest instance"; return PF_EINVAL; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (P.precision == PF_FP64) return run_batch_forked<double>(*D, R, s, err);
    return run_batch_forked<float>(*D, R, s, err);
}


// ------------------------------------------------------------------ tangents
// packed value state (phi, c, d) of the instances -> the Dual state of every
// (direction, instance) replica, derivative 0 (the initial fields do not
// depend on the parameters)
template <typename V>
__global__ void adjoint_replicate(const V* __restrict__ phi, const V* __restrict__ c, const V* __restrict__ d,
                                  long long total, int reps, Dual<V>* P, Dual<V>* Cc, Dual<V>* Dd) {
    const long long n = total * reps;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long s = k % total;
        P[k] = make_dual<V>(phi[s], V(0));
        Cc[k] = make_dual<V>(c[s], V(0));
        Dd[k] = make_dual<V>(d[s], V(0));
    }
}

// per replica: max_x c and the derivative of c at the maximising cell (lowest
// index among ties)
template <typename V>
__global__ void __launch_bounds__(256) adjoint_cmax(const Dual<V>* __restrict__ c, const BatchState* __restrict__ st,
                                                    double* __restrict__ out) {
    const BatchState S = st[blockIdx.x];
    double best = -INFINITY, tan = 0.0;
    int bi = 0x7fffffff;
    for (int i = threadIdx.x; i < S.n; i += blockDim.x) {
        const Dual<V> x = c[S.off + i];
        const double v = (double)x.v;
        if (v > best || (v == best && i < bi)) {
            best = v;
            tan = (double)x.t;
            bi = i;
        }
    }
    __shared__ double sb[256], st_[256];
    __shared__ int si[256];
    sb[threadIdx.x] = best;
    st_[threadIdx.x] = tan;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const double vb = sb[threadIdx.x + o];
            const int ib = si[threadIdx.x + o];
            if (vb > sb[threadIdx.x] || (vb == sb[threadIdx.x] && ib < si[threadIdx.x])) {
                sb[threadIdx.x] = vb;
                st_[threadIdx.x] = st_[threadIdx.x + o];
                si[threadIdx.x] = ib;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = sb[0];
        out[2 * blockIdx.x + 1] = st_[0];
    }
}

template <typename V>
static int run_adjoint_T(const pf_adjoint_desc& A, pf_adjoint_result* R, cudaStream_t main, std::string& err) {
    using T = Dual<V>;
    const pf_batch_desc& D = A.batch;
    const int N = D.n_instances;
    std::vector<int> dirs;
    for (int j = 0; j < 3; ++j)
        if ((A.wrt >> j) & 1) dirs.push_back(j);
    const int ND = (int)dirs.size();
    const int M = N * ND;
    // replicas r = q N + i: instance i, parameter dirs[q]
    std::vector<int64_t> rn(M);
    std::vector<double> rv(M), rdt(M);
    std::vector<int> rdir(M);
    std::vector<double> dt1;
    if (!batch_time_steps(D, dt1, err)) return PF_EINVAL;
    for (int q = 0; q < ND; ++q)
        for (int i = 0; i < N; ++i) {
            rn[q * N + i] = D.n[i];
            rv[q * N + i] = D.v_pull[i];
            rdt[q * N + i] = dt1[i];
            rdir[q * N + i] = dirs[q];
        }
    pf_batch_desc RD = D;
    RD.n_instances = M;
    RD.n = rn.data();
    RD.v_pull = rv.data();
    RD.dt = rdt.data();
    RD.check_every = 0;   // fixed number of steps, no convergence test
    RD.energy_every = 0;
    BatchRun<T> B(RD, main, err);
    B.rep_dir = rdir;
    B.off.resize(M);
    B.dt = rdt;
    int64_t total1 = 0;
    for (int i = 0; i < N; ++i) total1 += D.n[i];
    for (int r = 0; r < M; ++r) {
        B.off[r] = B.total;
        B.total += rn[r];
    }
    const size_t fb = (size_t)B.total * sizeof(T), vb = (size_t)total1 * sizeof(V);
    V *vphi = nullptr, *vcs = nullptr, *vcl = nullptr, *vc = nullptr, *vd = nullptr;
    double* dout = nullptr;
    cudaError_t e = cudaMalloc(&B.phi, fb);
    if (e == cudaSuccess) e = cudaMalloc(&B.c, fb);
    if (e == cudaSuccess) e = cudaMalloc(&B.d, fb);
    if (e == cudaSuccess) e = cudaMalloc(&B.st, M * sizeof(BatchState));
    if (e == cudaSuccess) e = cudaMalloc(&B.dv, M * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&B.ddt, M * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&vphi, vb);
    if (e == cudaSuccess) e = cudaMalloc(&vcs, vb);
    if (e == cudaSuccess) e = cudaMalloc(&vcl, vb);
    if (e == cudaSuccess) e = cudaMalloc(&vc, vb);
    if (e == cudaSuccess) e = cudaMalloc(&vd, vb);
    if (e == cudaSuccess) e = cudaMalloc(&dout, 2 * M * sizeof(double));
    auto free_tmp = [&] {
        void* ptrs[] = {vphi, vcs, vcl, vc, vd, dout};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    };
    if (e != cudaSuccess) {
        free_tmp();
        cudaGetLastError();
        err = std::string("device allocation failed: ") + cudaGetErrorString(e);
        return PF_ENOMEM;
    }
    std::vector<BatchState> hs(M);
    for (int r = 0; r < M; ++r) hs[r] = BatchState{B.off[r], (int)rn[r], 0, 0, 0, 0.0, 0.0, 0.0, 0.0};
    e = cudaMemcpyAsync(vphi, D.phi0, vb, cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vcs, D.cs0, vb, cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vcl, D.cl0, vb, cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.st, hs.data(), M * sizeof(BatchState), cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.dv, rv.data(), M * sizeof(double), cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.ddt, rdt.data(), M * sizeof(double), cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) {
        batch_to_state<V><<<1216, 256, 0, main>>>(vcs, vcl, vphi, vc, vd, total1, D.params.interp, D.params.a);
        adjoint_replicate<V><<<1216, 256, 0, main>>>(vphi, vc, vd, total1, ND, B.phi, B.c, B.d);
        e = cudaGetLastError();
    }
    size_t max_dyn = 0;
    if (e == cudaSuccess) e = set_smem_limits<T>(&max_dyn);
    if (e == cudaSuccess) {
        int64_t nbig = 0;
        for (int i = 0; i < N; ++i) nbig = std::max(nbig, (int64_t)D.n[i]);
        if ((size_t)6 * nbig * sizeof(T) > max_dyn) {
            free_tmp();
            err = "longest instance does not fit in shared memory";
            return PF_EINVAL;
        }
    }
    const int cpt = D.cells_per_thread > 0 ? D.cells_per_thread : 8;
    if (e == cudaSuccess) e = B.make_groups(cpt);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&B.t0);
    if (e == cudaSuccess) e = cudaEventCreate(&B.t1);
    const int64_t chunk = D.steps_per_launch > 0 ? D.steps_per_launch : A.nsteps;
    if (e == cudaSuccess) e = cudaEventRecord(B.t0, main);
    for (int64_t done = 0; done < A.nsteps && e == cudaSuccess; done += chunk)
        e = B.issue((int)std::min(chunk, A.nsteps - done));
    if (e == cudaSuccess) e = cudaEventRecord(B.t1, main);
    if (e == cudaSuccess) {
        adjoint_cmax<V><<<M, 256, 0, main>>>(B.c, B.st, dout);
        e = cudaGetLastError();
    }
    std::vector<double> hout(2 * M);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout.data(), dout, 2 * M * sizeof(double), cudaMemcpyDeviceToHost, main);
    if (e == cudaSuccess) e = cudaStreamSynchronize(main);
    float ms = 0;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, B.t0, B.t1);
    free_tmp();
    if (e != cudaSuccess) {
        err = std::string("adjoint run: ") + cudaGetErrorString(e);
        return PF_ECUDA;
    }
    // k_i = c_inf / c_max,i and dk_i = -c_inf dc_max,i / c_max,i^2; the loss
    const double cinf = D.params.c_inf;
    R->loss = 0.0;
    R->grad[0] = R->grad[1] = R->grad[2] = 0.0;
    for (int i = 0; i < N; ++i) {
        const double cm = hout[2 * i];
        const double k = cinf / cm;
        if (R->k) R->k[i] = k;
        double dk[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < ND; ++q) dk[dirs[q]] = -cinf * hout[2 * (q * N + i) + 1] / (cm * cm);
        if (R->dk)
            for (int j = 0; j < 3; ++j) R->dk[3 * i + j] = dk[j];
        if (A.k_target) {
            const double res = k - A.k_target[i];
            R->loss += res * res;
            for (int j = 0; j < 3; ++j) R->grad[j] += 2.0 * res * dk[j];
        }
    }
    R->gpu_ms = ms;
    return PF_OK;
}

// ---------------------------------------------------------------------------
// Reverse sweep (pf_adjoint, PF_ADJ_REVERSE): the adjoint of one fused 1D step
// of batch_kernel, applied backwards over recorded states.  lambda = dk/du for
// the state u = (phi, c, d) of one instance; the parameter derivatives collect
// dk/d(1/M_phi), dk/dA, dk/db from every use inside the step.

// p''(phi) (d/dphi of dp_of)
template <typename T>
__device__ __forceinline__ T d2p_of(const Consts<T>& C, T f) {
    const T g = f * (T(1) - f);
    const T d2h = C.dh1 + f * (T(2) * C.dh2 + f * (T(3) * C.dh3 + f * (T(4) * C.dh4)));
    const T s = T(1) - T(2) * f;
    const T dw = T(2) * g * s;
    return d2h + C.a * (T(2) * dw + (f - T(0.5)) * T(2) * (s * s - T(2) * g));
}

// adjoints of the inputs of face1 (and of A, b) from those of its outputs (gc, gd)
template <typename T>
struct FaceAdj {
    T f, cs, cl, pd;          // of each of the two cells' phi, c_s, c_l, phidot (half the face's)
    T nphi, nY, nS, nL;       // of the normal differences
    T A, b;                   // of the parameters
};

template <typename T>
__device__ void face1_rev(const Consts<T>& C, T fL, T fR, T csL, T csR, T clL, T clR, T pdL, T pdR,
                          T nphi, T nY, T nS, T nL, T gc, T gd, FaceAdj<T>& o) {
    // forward values (as face1)
    const T f = T(0.5) * (fL + fR);
    const T cs = T(0.5) * (csL + csR), cl = T(0.5) * (clL + clR);
    const T d = cs - cl;
    const T pdot = T(0.5) * (pdL + pdR);
    const T p = p_of(C, f);
    const T omp = T(1) - p;
    const T Ms = Ms_of(C, cs), Ml = Ml_of(C, cl);
    const T bMl = C.b * Ml;
    const T iM = T(1) / (Ms * omp + bMl * p);
    const T g2 = C.delta2;
    const T r = T(1) / (nphi * nphi + g2);
    const T Ts = Ms * nS * g2;
    const T Tl = Ml * nL * g2;
    const T at = C.one_m_A * d * pdot * nphi;
    const T u = C.b * p + omp;
    const T q = Ms * Ml * u * iM;
    const T ppo = p * omp;
    const T afn = (Ms - bMl) * ppo * iM;
    const T Ssum = q * nphi * nphi * nY + p * Ts + omp * Tl + at * afn;
    // reverse
    const T lr = gc * Ssum + gd * (Ts - Tl + at);
    const T lS = gc * r;
    const T lTs = lS * p + gd * r;
    const T lTl = lS * omp - gd * r;
    const T lat = lS * afn + gd * r;
    const T lq = lS * nphi * nphi * nY;
    T lnphi = lS * q * T(2) * nphi * nY;
    const T lnY = lS * q * nphi * nphi;
    T lp = lS * (Ts - Tl);
    const T lafn = lS * at;
    T lMs = lafn * ppo * iM;
    T lbMl = -lafn * ppo * iM;
    lp += lafn * (Ms - bMl) * (omp - p) * iM;
    T liM = lafn * (Ms - bMl) * ppo;
    lMs += lq * Ml * u * iM;
    T lMl = lq * Ms * u * iM;
    const T lu = lq * Ms * Ml * iM;
    liM += lq * Ms * Ml * u;
    lp += lu * (C.b - T(1));
    T lb = lu * p;
    const T ld = lat * C.one_m_A * pdot * nphi;
    const T lpdot = lat * C.one_m_A * d * nphi;
    lnphi += lat * C.one_m_A * d * pdot;
    const T lA = -lat * d * pdot * nphi;
    lMs += lTs * nS * g2;
    const T lnS = lTs * Ms * g2;
    lMl += lTl * nL * g2;
    const T lnL = lTl * Ml * g2;
    lnphi += lr * (-r * r) * (T(2) * nphi);
    const T lMb = -liM * iM * iM;
    lMs += lMb * omp;
    lp += lMb * (bMl - Ms);
    lbMl += lMb * p;
    lMl += lbMl * C.b;
    lb += lbMl * Ml;
    T lcs = lMs * C.Ms_c + ld;
    T lcl = lMl * C.Ml_c - ld;
    const T lf = lp * dp_of(C, f);
    o.f = T(0.5) * lf;
    o.cs = T(0.5) * lcs;
    o.cl = T(0.5) * lcl;
    o.pd = T(0.5) * lpdot;
    o.nphi = lnphi;
    o.nY = lnY;
    o.nS = lnS;
    o.nL = lnL;
    o.A = lA;
    o.b = lb;
}

template <typename T>
struct RevArgs {
    const T* rec;            // recorded states and intermediates of the segment (batch_kernel layout)
    long long rec_steps;
    T* lphi;                 // adjoint state, packed like the value state
    T* lc;
    T* ld;
    double* grad;            // [instance][3]: d k_i / d(1/M_phi, A, b), accumulated
    const BatchState* st0;   // per instance at the segment start (off, n, step, shifts)
    const double* v;
    const double* dt;
    int nsteps;              // steps of this segment (<= RMAX_SEG)
    Consts<T> C;
    double theta_ref, G_theta, x0;
    T gphi, gcs, gcl, gmus, gmul;   // Dirichlet (hot end) ghost
};

constexpr int RMAX_SEG = 1024;

template <typename T, int NT, int RJ>
__global__ void __launch_bounds__(NT, 1) reverse_kernel(RevArgs<T> a) {
    const int inst = blockIdx.x;
    const BatchState S0 = a.st0[inst];
    const int n = S0.n;
    const long long off = S0.off;
    const Consts<T>& C = a.C;
    extern __shared__ __align__(16) unsigned char smem[];
    T* sF = reinterpret_cast<T*>(smem);   // phi
    T* sCs = sF + n;                      // c_s
    T* sCl = sCs + n;                     // c_l
    T* sMs = sCl + n;                     // mu_s
    T* sMl = sMs + n;                     // mu_l
    T* sPd = sMl + n;                     // phidot
    T* sLf = sPd + n;                     // adjoints of phi, c, d
    T* sLc = sLf + n;
    T* sLd = sLc + n;
    T* sXl = sLd + n;                     // per cell: adjoints of its rate's lap, d_x phi, d_x mu_s, d_x mu_l
    T* sXg = sXl + n;
    T* sXs = sXg + n;
    T* sXm = sXs + n;
    __shared__ int nsh[RMAX_SEG];         // window shifts that followed each step
    __shared__ double th0[RMAX_SEG];      // theta0 of each step
    __shared__ double red[NT / 32];
    const int tid = threadIdx.x;
    const double v = a.v[inst];
    const double dtd = a.dt[inst];
    const T dt = T(dtd);
    const T dtdx = dt * C.inv_dx;
    if (tid == 0) {   // replay the clock of batch_kernel over the segment
        long long step = S0.step, shifts = S0.shifts;
        for (int it = 0; it < a.nsteps; ++it) {
            th0[it] = a.theta_ref + a.G_theta * (a.x0 + v * ((double)step * dtd) - (double)shifts * (double)C.dx);
            step += 1;
            const double tn = (double)step * dtd;
            int k = 0;
            while (v * tn >= (double)(shifts + 1) * (double)C.dx) {
                shifts += 1;
                k += 1;
            }
            nsh[it] = k;
        }
    }
    for (int i = tid; i < n; i += NT) {
        sLf[i] = a.lphi[off + i];
        sLc[i] = a.lc[off + i];
        sLd[i] = a.ld[off + i];
    }
    __syncthreads();
    double gM = 0.0, gA = 0.0, gB = 0.0;
    const T pg = p_of(C, a.gphi);
    const T Yg = a.gmul + pg * (a.gmus - a.gmul);

    for (int it = a.nsteps - 1; it >= 0; --it) {
        // the window shifts after this step, undone: lambda moves one cell back
        for (int k = 0; k < nsh[it]; ++k) {
            T tf[RJ], tc[RJ], td[RJ];
#pragma unroll
            for (int j = 0; j < RJ; ++j) {
                const int i = tid + j * NT;
                if (i >= n) break;
                tf[j] = i > 0 ? sLf[i - 1] : T(0);
                tc[j] = i > 0 ? sLc[i - 1] : T(0);
                td[j] = i > 0 ? sLd[i - 1] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < RJ; ++j) {
                const int i = tid + j * NT;
                if (i >= n) break;
                sLf[i] = tf[j];
                sLc[i] = tc[j];
                sLd[i] = td[j];
            }
            __syncthreads();
        }
        // the step's state and intermediates, as the forward run recorded them
        const T* r = a.rec + 6 * a.rec_steps * off + (long long)it * 6 * n;
        T dval[RJ], pval[RJ];
#pragma unroll
        for (int j = 0; j < RJ; ++j) {
            const int i = tid + j * NT;
            if (i >= n) break;
            const T f = r[i], c = r[n + i], d = r[2 * n + i];
            const T p = p_of(C, f);
            sF[i] = f;
            sCs[i] = c + (T(1) - p) * d;
            sCl[i] = c - p * d;
            sMs[i] = r[3 * n + i];
            sMl[i] = r[4 * n + i];
            sPd[i] = r[5 * n + i];
            dval[j] = d;
            pval[j] = p;
        }
        __syncthreads();
        const T theta0 = T(th0[it]);
        // R1: the two faces of each cell, their parts that act on the cell
        T aF[RJ], aCs[RJ], aCl[RJ], aMs[RJ], aMl[RJ], aP[RJ], aPd[RJ];
#pragma unroll
        for (int j = 0; j < RJ; ++j) {
            const int i = tid + j * NT;
            if (i >= n) break;
            const T f0 = sF[i], cs0 = sCs[i], cl0 = sCl[i], ms0 = sMs[i], ml0 = sMl[i], pd0 = sPd[i];
            const T p0 = pval[j];
            const T Y0 = ml0 + p0 * (ms0 - ml0);
            T lf = T(0), lcs = T(0), lcl = T(0), lms = T(0), lml = T(0), lY = T(0);
            T lpd = dt * sLf[i];
            FaceAdj<T> o;
            if (i > 0) {   // face (i-1, i): this cell is its right side
                const T fL = sF[i - 1], csL = sCs[i - 1], clL = sCl[i - 1], msL = sMs[i - 1], mlL = sMl[i - 1];
                const T pL = p_of(C, fL);
                const T YL = mlL + pL * (msL - mlL);
                const T gc = dtdx * (sLc[i - 1] - sLc[i]), gd = dtdx * (sLd[i - 1] - sLd[i]);
                face1_rev(C, fL, f0, csL, cs0, clL, cl0, sPd[i - 1], pd0, (f0 - fL) * C.inv_dx,
                          (Y0 - YL) * C.inv_dx, (ms0 - msL) * C.inv_dx, (ml0 - mlL) * C.inv_dx, gc, gd, o);
                lf += o.f + o.nphi * C.inv_dx;
                lcs += o.cs;
                lcl += o.cl;
                lpd += o.pd;
                lY += o.nY * C.inv_dx;
                lms += o.nS * C.inv_dx;
                lml += o.nL * C.inv_dx;
            }
            {              // face (i, i+1), or (n-1, ghost): this cell is its left side
                const bool last = i == n - 1;
                const T fR = last ? a.gphi : sF[i + 1];
                const T csR = last ? a.gcs : sCs[i + 1], clR = last ? a.gcl : sCl[i + 1];
                const T msR = last ? a.gmus : sMs[i + 1], mlR = last ? a.gmul : sMl[i + 1];
                const T YR = last ? Yg : mlR + p_of(C, fR) * (msR - mlR);
                const T pdR = last ? T(0) : sPd[i + 1];
                const T gc = dtdx * (sLc[i] - (last ? T(0) : sLc[i + 1]));
                const T gd = dtdx * (sLd[i] - (last ? T(0) : sLd[i + 1]));
                face1_rev(C, f0, fR, cs0, csR, cl0, clR, pd0, pdR, (fR - f0) * C.inv_dx,
                          (YR - Y0) * C.inv_dx, (msR - ms0) * C.inv_dx, (mlR - ml0) * C.inv_dx, gc, gd, o);
                lf += o.f - o.nphi * C.inv_dx;
                lcs += o.cs;
                lcl += o.cl;
                lpd += o.pd;
                lY -= o.nY * C.inv_dx;
                lms -= o.nS * C.inv_dx;
                lml -= o.nL * C.inv_dx;
                gA += (double)o.A;   // each face's parameter terms counted once, by its left cell
                gB += (double)o.b;
            }
            // Y = mu_l + p (mu_s - mu_l)
            lms += lY * p0;
            lml += lY * (T(1) - p0);
            aP[j] = lY * (ms0 - ml0);
            aF[j] = lf;
            aCs[j] = lcs;
            aCl[j] = lcl;
            aMs[j] = lms;
            aMl[j] = lml;
            aPd[j] = lpd;
        }
        // R2: the phase-field rate of each cell, backwards
#pragma unroll
        for (int j = 0; j < RJ; ++j) {
            const int i = tid + j * NT;
            if (i >= n) break;
            const int im = (i == 0) ? 0 : i - 1;
            const bool last = i == n - 1;
            const T fc = sF[i], fW = sF[im], fE = last ? a.gphi : sF[i + 1];
            const T mWs = sMs[im], mWl = sMl[im];
            const T mEs = last ? a.gmus : sMs[i + 1], mEl = last ? a.gmul : sMl[i + 1];
            const T p = pval[j], cs = sCs[i], cl = sCl[i], mus = sMs[i], mul = sMl[i];
            const T dp = dp_of(C, fc);
            const T lap = (fW - T(2) * fc + fE) * C.inv_dx2;
            const T gp = (fE - fW) * C.inv_2dx;
            const T gs = (mEs - mWs) * C.inv_2dx;
            const T gl = (mEl - mWl) * C.inv_2dx;
            const T Ms = Ms_of(C, cs), Ml = Ml_of(C, cl);
            const T bMl = C.b * Ml;
            const T omp = T(1) - p;
            const T Msq = Ms * omp;
            const T iM = T(1) / (Msq + bMl * p);
            const T d = cs - cl;
            const T rr = T(1) / (gp * gp + C.delta2);
            const T pq = p * omp;
            const T u = C.b * p + omp;
            const T oA = C.one_m_A;
            const T K2 = oA * oA * d * d * C.b * pq * rr * iM / u;
            const T Kc = C.inv_Mphi + K2;
            const T theta = theta0 - C.G_theta * ((T(i) + T(0.5)) * C.dx);
            const T dmu = mus - mul;
            const T Nv = Msq * (T(1) - C.A * omp) + C.A * bMl * p * p;
            const T Dd = Nv * iM;
            const T dG = cs * dmu - d - C.one_m_ke * theta - Dd * d * dmu;
            const T W = Ms * gs - bMl * gl;
            const T Xv = W * gp * rr;
            const T pd = sPd[i];
            const T lpd = aPd[j];
            const T lR = lpd / Kc;
            const T lKc = -lpd * pd / Kc;
            const T llap = lR * C.sigma;
            const T ldfdw = -lR * C.H;
            const T ldG = -lR * dp;
            const T ldp = -lR * dG;
            // Z = (1-A) d pq iM X
            T loA = lR * d * pq * iM * Xv;
            T ld = lR * oA * pq * iM * Xv;
            T lpq = lR * oA * d * iM * Xv;
            T liM = lR * oA * d * pq * Xv;
            const T lX = lR * oA * d * pq * iM;
            const T lW = lX * gp * rr;
            T lgp = lX * W * rr;
            T lrr = lX * W * gp;
            T lMs = lW * gs;
            const T lgs = lW * Ms;
            T lbMl = -lW * gl;
            const T lgl = -lW * bMl;
            // Kc = 1/M_phi + (1-A)^2 d^2 b pq rr iM / u
            gM += (double)lKc;
            loA += lKc * T(2) * oA * d * d * C.b * pq * rr * iM / u;
            ld += lKc * oA * oA * T(2) * d * C.b * pq * rr * iM / u;
            T lb = lKc * oA * oA * d * d * pq * rr * iM / u;
            lpq += lKc * oA * oA * d * d * C.b * rr * iM / u;
            lrr += lKc * oA * oA * d * d * C.b * pq * iM / u;
            liM += lKc * oA * oA * d * d * C.b * pq * rr / u;
            const T lu = -lKc * K2 / u;
            T lp = lu * (C.b - T(1));
            lb += lu * p;
            // dG = cs dmu - d - (1-k_e) theta - Dd d dmu
            T lcs = ldG * dmu;
            const T ldmu = ldG * (cs - Dd * d);
            ld += -ldG * (T(1) + Dd * dmu);
            const T lDd = -ldG * d * dmu;
            // Dd = Nv iM
            const T lN = lDd * iM;
            liM += lDd * Nv;
            T lMsq = lN * (T(1) - C.A * omp);
            gA += (double)(lN * (-Msq * omp + bMl * p * p));
            lp += lN * (Msq * C.A + T(2) * C.A * bMl * p);
            lbMl += lN * C.A * p * p;
            // dmu, pq, rr, iM, Msq, bMl, Ms, Ml, d
            const T lmus = ldmu, lmul = -ldmu;
            lp += lpq * (T(1) - T(2) * p);
            lgp += lrr * (-rr * rr) * (T(2) * gp);
            const T lden = -liM * iM * iM;
            lMsq += lden;
            lbMl += lden * p;
            lp += lden * bMl;
            lMs += lMsq * omp;
            lp -= lMsq * Ms;
            T lMl = lbMl * C.b;
            lb += lbMl * Ml;
            lcs += lMs * C.Ms_c + ld;
            T lcl = lMl * C.Ml_c - ld;
            gA -= (double)loA;   // one_m_A = 1 - A
            gB += (double)lb;
            // phi of the cell itself: f_dw', p', the Laplacian's centre (and its own
            // west neighbour at the mirrored cold end)
            T lf = ldfdw * T(2) * (T(1) - T(6) * fc + T(6) * fc * fc) + ldp * d2p_of(C, fc)
                   - T(2) * llap * C.inv_dx2;
            T lms_self = lmus, lml_self = lmul;
            if (i == 0) {
                lf += llap * C.inv_dx2 - lgp * C.inv_2dx;
                lms_self -= lgs * C.inv_2dx;
                lml_self -= lgl * C.inv_2dx;
            }
            aF[j] += lf;
            aCs[j] += lcs;
            aCl[j] += lcl;
            aMs[j] += lms_self;
            aMl[j] += lml_self;
            aP[j] += lp;
            sXl[i] = llap;
            sXg[i] = lgp;
            sXs[i] = lgs;
            sXm[i] = lgl;
        }
        __syncthreads();
        // R3: the neighbours' rates, then the pointwise values, into the adjoint
        // of the pre-step state (in place: R3 reads only its own cells' lambda)
#pragma unroll
        for (int j = 0; j < RJ; ++j) {
            const int i = tid + j * NT;
            if (i >= n) break;
            T lf = aF[j], lms = aMs[j], lml = aMl[j];
            if (i > 0) {        // this cell is the east neighbour of cell i-1
                lf += sXl[i - 1] * C.inv_dx2 + sXg[i - 1] * C.inv_2dx;
                lms += sXs[i - 1] * C.inv_2dx;
                lml += sXm[i - 1] * C.inv_2dx;
            }
            if (i < n - 1) {    // and the west neighbour of cell i+1
                lf += sXl[i + 1] * C.inv_dx2 - sXg[i + 1] * C.inv_2dx;
                lms -= sXs[i + 1] * C.inv_2dx;
                lml -= sXm[i + 1] * C.inv_2dx;
            }
            const T cs = sCs[i], cl = sCl[i];
            const T lcs = aCs[j] + lms / cs;
            const T lcl = aCl[j] + lml / cl;
            const T p = pval[j];
            const T lp = aP[j] - dval[j] * (lcs + lcl);
            sLf[i] = sLf[i] + lf + lp * dp_of(C, sF[i]);
            sLc[i] = sLc[i] + lcs + lcl;
            sLd[i] = sLd[i] + lcs * (T(1) - p) - lcl * p;
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += NT) {
        a.lphi[off + i] = sLf[i];
        a.lc[off + i] = sLc[i];
        a.ld[off + i] = sLd[i];
    }
    // parameter derivatives: block sums, one writer per instance
    double vals[3] = {gM, gA, gB};
    for (int q = 0; q < 3; ++q) {
        double x = vals[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((tid & 31) == 0) red[tid >> 5] = x;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < NT / 32; ++w) tot += red[w];
            a.grad[3 * inst + q] += tot;
        }
        __syncthreads();
    }
}

// per instance: max_x c and the lowest maximising index
template <typename V>
__global__ void __launch_bounds__(256) value_cmax(const V* __restrict__ c, const BatchState* __restrict__ st,
                                                  double* __restrict__ cmax, int* __restrict__ imax) {
    const BatchState S = st[blockIdx.x];
    double best = -INFINITY;
    int bi = 0x7fffffff;
    for (int i = threadIdx.x; i < S.n; i += blockDim.x) {
        const double x = (double)c[S.off + i];
        if (x > best || (x == best && i < bi)) {
            best = x;
            bi = i;
        }
    }
    __shared__ double sb[256];
    __shared__ int si[256];
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const double vb = sb[threadIdx.x + o];
            const int ib = si[threadIdx.x + o];
            if (vb > sb[threadIdx.x] || (vb == sb[threadIdx.x] && ib < si[threadIdx.x])) {
                sb[threadIdx.x] = vb;
                si[threadIdx.x] = ib;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        cmax[blockIdx.x] = sb[0];
        imax[blockIdx.x] = si[0];
    }
}

// lambda at the end of the run: d k_i / d c at the maximising cell, -c_inf / c_max^2
template <typename V>
__global__ void seed_lambda(V* __restrict__ lc, const BatchState* __restrict__ st, const double* __restrict__ cmax,
                            const int* __restrict__ imax, double cinf, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // a run that went non-finite has no maximising cell: nothing is seeded (k is NaN)
    if (i < N && imax[i] >= 0 && imax[i] < st[i].n) lc[st[i].off + imax[i]] = V(-cinf / (cmax[i] * cmax[i]));
}

// 512 threads per instance, RJ cells each: the smallest RJ that covers the
// longest instance (registers hold RJ cells' partial adjoints)
template <typename V>
using RevFn = void (*)(RevArgs<V>);
template <typename V>
static RevFn<V> reverse_for(int64_t nmax) {
    if (nmax <= 1024) return reverse_kernel<V, 512, 2>;
    if (nmax <= 2048) return reverse_kernel<V, 512, 4>;
    return reverse_kernel<V, 512, 8>;
}

template <typename V>
static int run_adjoint_reverse_T(const pf_adjoint_desc& A, pf_adjoint_result* R, cudaStream_t main, std::string& err) {
    constexpr int NT = 512;
    pf_batch_desc D = A.batch;
    D.check_every = 0;   // a fixed number of steps
    D.energy_every = 0;
    const int N = D.n_instances;
    BatchRun<V> B(D, main, err);
    B.off.resize(N);
    for (int i = 0; i < N; ++i) {
        B.off[i] = B.total;
        B.total += D.n[i];
    }
    if (!batch_time_steps(D, B.dt, err)) return PF_EINVAL;
    int64_t nmax = 0;
    for (int i = 0; i < N; ++i) nmax = std::max(nmax, (int64_t)D.n[i]);
    const int64_t seg = std::min<int64_t>(
        {A.checkpoint_every > 0 ? (int64_t)A.checkpoint_every
                                : (int64_t)std::ceil(std::sqrt((double)A.nsteps)),
         (int64_t)RMAX_SEG, A.nsteps});
    const int64_t nseg = (A.nsteps + seg - 1) / seg;
    const size_t fb = (size_t)B.total * sizeof(V);
    V *scs = nullptr, *scl = nullptr, *ckp = nullptr, *ckc = nullptr, *ckd = nullptr, *rec = nullptr;
    V *lphi = nullptr, *lc = nullptr, *ld = nullptr;
    BatchState* ckst = nullptr;
    double *grad = nullptr, *cmax = nullptr;
    int* imax = nullptr;
    auto free_tmp = [&] {
        void* ptrs[] = {scs, scl, ckp, ckc, ckd, rec, lphi, lc, ld, ckst, grad, cmax, imax};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    };
    cudaError_t e = cudaMalloc(&B.phi, fb);
    if (e == cudaSuccess) e = cudaMalloc(&B.c, fb);
    if (e == cudaSuccess) e = cudaMalloc(&B.d, fb);
    if (e == cudaSuccess) e = cudaMalloc(&B.st, N * sizeof(BatchState));
    if (e == cudaSuccess) e = cudaMalloc(&B.dv, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&B.ddt, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&scs, fb);
    if (e == cudaSuccess) e = cudaMalloc(&scl, fb);
    if (e == cudaSuccess) e = cudaMalloc(&ckp, fb * nseg);
    if (e == cudaSuccess) e = cudaMalloc(&ckc, fb * nseg);
    if (e == cudaSuccess) e = cudaMalloc(&ckd, fb * nseg);
    if (e == cudaSuccess) e = cudaMalloc(&ckst, (size_t)N * nseg * sizeof(BatchState));
    if (e == cudaSuccess) e = cudaMalloc(&rec, fb * 6 * seg * 2);
    if (e == cudaSuccess) e = cudaMalloc(&lphi, fb);
    if (e == cudaSuccess) e = cudaMalloc(&lc, fb);
    if (e == cudaSuccess) e = cudaMalloc(&ld, fb);
    if (e == cudaSuccess) e = cudaMalloc(&grad, 3 * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&cmax, N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&imax, N * sizeof(int));
    if (e != cudaSuccess) {
        free_tmp();
        cudaGetLastError();
        err = std::string("device allocation failed: ") + cudaGetErrorString(e);
        return PF_ENOMEM;
    }
    std::vector<BatchState> hs(N);
    for (int i = 0; i < N; ++i) hs[i] = BatchState{B.off[i], (int)D.n[i], 0, 0, 0, 0.0, 0.0, 0.0, 0.0};
    e = cudaMemcpyAsync(B.phi, D.phi0, fb, cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scs, D.cs0, fb, cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scl, D.cl0, fb, cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.st, hs.data(), N * sizeof(BatchState), cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.dv, D.v_pull, N * sizeof(double), cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.ddt, B.dt.data(), N * sizeof(double), cudaMemcpyHostToDevice, main);
    if (e == cudaSuccess) e = cudaMemsetAsync(lphi, 0, fb, main);
    if (e == cudaSuccess) e = cudaMemsetAsync(lc, 0, fb, main);
    if (e == cudaSuccess) e = cudaMemsetAsync(ld, 0, fb, main);
    if (e == cudaSuccess) e = cudaMemsetAsync(grad, 0, 3 * N * sizeof(double), main);
    if (e == cudaSuccess) {
        batch_to_state<V><<<1216, 256, 0, main>>>(scs, scl, B.phi, B.c, B.d, B.total, D.params.interp, D.params.a);
        e = cudaGetLastError();
    }
    size_t max_dyn = 0;
    if (e == cudaSuccess) e = set_smem_limits<V>(&max_dyn);
    const size_t rsmem = (size_t)13 * nmax * sizeof(V);
    if (e == cudaSuccess) {
        static DeviceSetup setup;
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess && (dev < 0 || dev >= DeviceSetup::MAX_DEVICES)) e = cudaErrorInvalidDevice;
        if (e == cudaSuccess) {
            std::lock_guard<std::mutex> lock(setup.mu);
            if (!setup.done[dev]) {
                int optin = 0;
                setup.err[dev] = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
                for (int64_t m : {int64_t(1024), int64_t(2048), int64_t(4096)})
                    if (setup.err[dev] == cudaSuccess) setup.err[dev] = raise_smem(reverse_for<V>(m), optin);
                cudaFuncAttributes fa;
                if (setup.err[dev] == cudaSuccess) setup.err[dev] = cudaFuncGetAttributes(&fa, reverse_for<V>(4096));
                setup.value[dev] = setup.err[dev] == cudaSuccess ? (size_t)optin - fa.sharedSizeBytes : 0;
                setup.done[dev] = true;
            }
            e = setup.err[dev];
            if (e == cudaSuccess && rsmem > setup.value[dev]) {
                free_tmp();
                err = "longest instance does not fit in shared memory for the reverse sweep";
                return PF_EINVAL;
            }
        }
    }
    if (e == cudaSuccess && (size_t)6 * nmax * sizeof(V) > max_dyn) {
        free_tmp();
        err = "longest instance does not fit in shared memory";
        return PF_EINVAL;
    }
    const int cpt = D.cells_per_thread > 0 ? D.cells_per_thread : 8;
    if (e == cudaSuccess) e = B.make_groups(cpt);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&B.t0);
    if (e == cudaSuccess) e = cudaEventCreate(&B.t1);
    if (e == cudaSuccess) e = cudaEventRecord(B.t0, main);
    // forward: the state (and clock) before every segment, then the segment
    for (int64_t s = 0; s < nseg && e == cudaSuccess; ++s) {
        const int64_t len = std::min(seg, A.nsteps - s * seg);
        e = cudaMemcpyAsync(ckp + s * B.total, B.phi, fb, cudaMemcpyDeviceToDevice, main);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ckc + s * B.total, B.c, fb, cudaMemcpyDeviceToDevice, main);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ckd + s * B.total, B.d, fb, cudaMemcpyDeviceToDevice, main);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ckst + s * N, B.st, N * sizeof(BatchState), cudaMemcpyDeviceToDevice, main);
        if (e == cudaSuccess) e = B.issue((int)len);
    }
    if (e == cudaSuccess) {
        value_cmax<V><<<N, 256, 0, main>>>(B.c, B.st, cmax, imax);
        seed_lambda<V><<<(N + 255) / 256, 256, 0, main>>>(lc, B.st, cmax, imax, D.params.c_inf, N);
        e = cudaGetLastError();
    }
    // backwards: re-run each segment recording every step (main stream, the
    // batch kernel) and sweep it (a second stream, the reverse kernel).  The
    // records are double-buffered, so the re-run of segment s-1 overlaps the
    // sweep of segment s; the sweeps run in order on their stream.
    cudaStream_t rs = nullptr;
    cudaEvent_t erec[2] = {nullptr, nullptr}, erev[2] = {nullptr, nullptr};
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&erec[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&erev[b], cudaEventDisableTiming);
    }
    B.rec_steps = seg;
    const size_t rec_elems = (size_t)6 * seg * B.total;
    auto rerun = [&](int64_t s) {
        const int b = (int)(s & 1);
        const int64_t len = std::min(seg, A.nsteps - s * seg);
        cudaError_t x = cudaSuccess;
        if (s + 2 < nseg) x = cudaStreamWaitEvent(main, erev[b], 0);   // the sweep of s+2 read this buffer
        if (x == cudaSuccess) x = cudaMemcpyAsync(B.phi, ckp + s * B.total, fb, cudaMemcpyDeviceToDevice, main);
        if (x == cudaSuccess) x = cudaMemcpyAsync(B.c, ckc + s * B.total, fb, cudaMemcpyDeviceToDevice, main);
        if (x == cudaSuccess) x = cudaMemcpyAsync(B.d, ckd + s * B.total, fb, cudaMemcpyDeviceToDevice, main);
        if (x == cudaSuccess)
            x = cudaMemcpyAsync(B.st, ckst + s * N, N * sizeof(BatchState), cudaMemcpyDeviceToDevice, main);
        B.rec = rec + b * rec_elems;
        if (x == cudaSuccess) x = B.issue((int)len);
        if (x == cudaSuccess) x = cudaEventRecord(erec[b], main);
        return x;
    };
    if (e == cudaSuccess) e = rerun(nseg - 1);
    for (int64_t s = nseg - 1; s >= 0 && e == cudaSuccess; --s) {
        const int b = (int)(s & 1);
        const int64_t len = std::min(seg, A.nsteps - s * seg);
        e = cudaStreamWaitEvent(rs, erec[b], 0);
        if (e == cudaSuccess) {
            const BatchArgs<V> ba = B.args(B.groups[0], (int)len);
            RevArgs<V> ra;
            ra.rec = rec + b * rec_elems;
            ra.rec_steps = seg;
            ra.lphi = lphi;
            ra.lc = lc;
            ra.ld = ld;
            ra.grad = grad;
            ra.st0 = ckst + s * N;
            ra.v = B.dv;
            ra.dt = B.ddt;
            ra.nsteps = (int)len;
            ra.C = ba.C;
            ra.theta_ref = ba.theta_ref;
            ra.G_theta = ba.G_theta;
            ra.x0 = ba.x0;
            ra.gphi = ba.gphi;
            ra.gcs = ba.gcs;
            ra.gcl = ba.gcl;
            ra.gmus = ba.gmus;
            ra.gmul = ba.gmul;
            reverse_for<V>(nmax)<<<N, NT, rsmem, rs>>>(ra);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(erev[b], rs);
        if (e == cudaSuccess && s > 0) e = rerun(s - 1);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(main, erev[0], 0);   // the sweep of segment 0
    if (rs) {
        cudaStreamSynchronize(rs);
        cudaStreamDestroy(rs);
    }
    for (int b = 0; b < 2; ++b) {
        if (erec[b]) cudaEventDestroy(erec[b]);
        if (erev[b]) cudaEventDestroy(erev[b]);
    }
    if (e == cudaSuccess) e = cudaEventRecord(B.t1, main);
    std::vector<double> hg(3 * N), hc(N);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hg.data(), grad, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, main);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), cmax, N * sizeof(double), cudaMemcpyDeviceToHost, main);
    if (e == cudaSuccess) e = cudaStreamSynchronize(main);
    float ms = 0;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, B.t0, B.t1);
    free_tmp();
    if (e != cudaSuccess) {
        err = std::string("reverse adjoint run: ") + cudaGetErrorString(e);
        return PF_ECUDA;
    }
    const double cinf = D.params.c_inf, Mphi = D.params.M_phi;
    R->loss = 0.0;
    R->grad[0] = R->grad[1] = R->grad[2] = 0.0;
    for (int i = 0; i < N; ++i) {
        const double k = cinf / hc[i];
        if (R->k) R->k[i] = k;
        // d k / d(1/M_phi) -> d k / d M_phi
        const double all[3] = {hg[3 * i] * (-1.0 / (Mphi * Mphi)), hg[3 * i + 1], hg[3 * i + 2]};
        double dk[3];
        for (int j = 0; j < 3; ++j) dk[j] = ((A.wrt >> j) & 1) ? all[j] : 0.0;
        if (R->dk)
            for (int j = 0; j < 3; ++j) R->dk[3 * i + j] = dk[j];
        if (A.k_target) {
            const double res = k - A.k_target[i];
            R->loss += res * res;
            for (int j = 0; j < 3; ++j) R->grad[j] += 2.0 * res * dk[j];
        }
    }
    R->gpu_ms = ms;
    return PF_OK;
}

int run_adjoint(const pf_adjoint_desc* A, pf_adjoint_result* R, void* stream, std::string& err) {
    if (!A || !R) { err = "null argument"; return PF_EINVAL; }
    const pf_batch_desc& D = A->batch;
    const pf_params& P = D.params;
    if (A->nsteps <= 0 || A->nsteps > (int64_t(1) << 40)) { err = "nsteps must be positive"; return PF_EINVAL; }
    if (A->wrt <= 0 || A->wrt > 7) { err = "wrt must be a non-empty set of PF_ADJ_* bits"; return PF_EINVAL; }
    if (A->mode != PF_ADJ_TANGENT && A->mode != PF_ADJ_REVERSE) { err = "mode must be PF_ADJ_TANGENT or PF_ADJ_REVERSE"; return PF_EINVAL; }
    if (A->checkpoint_every < 0) { err = "checkpoint_every must be >= 0"; return PF_EINVAL; }
    const int64_t nmax = (P.precision == PF_FP64) ? 2048 : 4096;
    if (D.n_instances <= 0 || !D.n || !D.v_pull || !D.phi0 || !D.cs0 || !D.cl0) { err = "empty batch or null array"; return PF_EINVAL; }
    for (int i = 0; i < D.n_instances; ++i) {
        if (D.n[i] < 8 || D.n[i] > nmax) { err = "instance length outside 8.." + std::to_string(nmax); return PF_EINVAL; }
        if (!(D.v_pull[i] >= 0) || !std::isfinite(D.v_pull[i])) { err = "negative or non-finite velocity"; return PF_EINVAL; }
    }
    if (!(D.dx > 0) || !(P.k_e > 0 && P.k_e < 1) || !(P.b > 0) || !(P.M_phi > 0) || !(P.H > 0) ||
        !(P.sigma > 0) || !(P.D_s > 0) || !(P.D_l > 0) || !(P.c_inf > 0)) {
        err = "invalid model parameters";
        return PF_EINVAL;
    }
    if (P.precision != PF_FP32 && P.precision != PF_FP64) { err = "precision must be PF_FP32 or PF_FP64"; return PF_EINVAL; }
    if (D.bc.lo[0] != PF_BC_NOFLUX || D.bc.hi[0] != PF_BC_DIRICHLET) {
        err = "instances need a no-flux cold end and a Dirichlet hot end";
        return PF_EINVAL;
    }
    if (!(D.bc.dir_cs > 0) || !(D.bc.dir_cl > 0)) { err = "Dirichlet concentrations must be positive"; return PF_EINVAL; }
    const int cpt = D.cells_per_thread;
    if (cpt != 0 && cpt != 1 && cpt != 2 && cpt != 4 && cpt != 8) { err = "cells_per_thread must be 0, 1, 2, 4 or 8"; return PF_EINVAL; }
    for (int i = 0; i < D.n_instances; ++i)
        if (D.n[i] > (int64_t)1024 * (cpt > 0 ? cpt : 8)) { err = "cells_per_thread too small for the longest instance"; return PF_EINVAL; }
    if (D.steps_per_launch < 0 || D.steps_per_launch > (1 << 30)) { err = "steps_per_launch must be in 0..2^30"; return PF_EINVAL; }
    if (D.steps_per_launch == 0 && A->nsteps > (1 << 30)) { err = "nsteps above 2^30 needs steps_per_launch"; return PF_EINVAL; }
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    cudaStream_t work = nullptr;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&work, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(work, ev, 0);
    int rc = PF_ECUDA;
    if (e == cudaSuccess) {
        if (A->mode == PF_ADJ_REVERSE)
            rc = (P.precision == PF_FP64) ? run_adjoint_reverse_T<double>(*A, R, work, err)
                                          : run_adjoint_reverse_T<float>(*A, R, work, err);
        else
            rc = (P.precision == PF_FP64) ? run_adjoint_T<double>(*A, R, work, err) : run_adjoint_T<float>(*A, R, work, err);
        cudaError_t e2 = cudaEventRecord(ev, work);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(caller, ev, 0);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(work);
        if (rc == PF_OK && e2 != cudaSuccess) {
            err = std::string("adjoint join: ") + cudaGetErrorString(e2);
            rc = PF_ECUDA;
        }
    } else {
        err = std::string("adjoint stream: ") + cudaGetErrorString(e);
    }
    if (ev) cudaEventDestroy(ev);
    if (work) cudaStreamDestroy(work);
    return rc;
}

}  // namespace pf

namespace {
thread_local std::string g_batch_error;
}

extern "C" int pf_run_batch(const pf_batch_desc* desc, pf_batch_result* res, void* stream) {
    g_batch_error.clear();
    const int rc = pf::run_batch(desc, res, stream, g_batch_error);
    if (rc != PF_OK) pf::set_create_error(g_batch_error);
    return rc;
}

extern "C" int pf_adjoint(const pf_adjoint_desc* desc, pf_adjoint_result* res, void* stream) {
    g_batch_error.clear();
    const int rc = pf::run_adjoint(desc, res, stream, g_batch_error);
    if (rc != PF_OK) pf::set_create_error(g_batch_error);
    return rc;
}
