// pf_kernels.h -- host-side launch interface between the C ABI (pf_api.cu)
// and the kernels (pf_step.cu, pf_diag.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cmath>
#include <mutex>
#include <string>
#include <cuda_runtime.h>
#include "pf.h"

namespace pf {

// Validated problem description, host copy (FP64 parameters).
struct HostProblem {
    int dim;
    int64_t n[3];
    double dx;
    int bc_lo[3], bc_hi[3];
    double dir_phi, dir_cs, dir_cl;
    int precision;   // 0 FP32, 1 FP64
    int interp, lap, mobility;
    double H, sigma, M_phi, D_s, D_l, k_e, A, b, a, delta;
    double theta_ref, G_theta, v_pull, x0, dt, c_inf;
    int shift;
    int64_t cells() const { return n[0] * n[1] * n[2]; }
    size_t elem() const { return precision == 1 ? sizeof(double) : sizeof(float); }
};

// Device state: phi, c = p c_s + (1-p) c_l, d = c_s - c_l and, in FP32, the
// low word c_lo of c (NULL in FP64).  A 1D FP32 state also keeps the low word
// phi_lo of phi (NULL otherwise): there the rounding of phi to FP32 after
// every step, accumulated over the slow motion of a planar front, is the
// largest FP32 error.
struct Fields {
    void *phi, *c, *d, *clo, *plo;
};

struct StepLaunch {
    const HostProblem* prob;
    const void *phi_in, *c_in, *d_in, *clo_in, *plo_in;
    void *phi_out, *c_out, *d_out, *clo_out, *plo_out;
    int64_t step, shifts;   // clock of the input state
    int zchunk;             // planes per CTA along z (3D); <= 0: automatic
    int zfirst = 0, zcount = 0;   // 3D: run z-chunks [zfirst, zfirst + zcount) only; zcount <= 0: all
    bool use_generic;       // 2D / 3D: the generic (1D/2D/3D) kernel instead of the paired one
    cudaStream_t stream;
    int* err = nullptr;     // device flag a step kernel sets when a bounded wait runs out (or NULL)
    bool no_tma = false;    // 3D: per-cell cp.async plane loads even where TMA boxes apply
    bool drop_copies = false;   // 3D TMA: arrive without issuing the copies (tests the bounded wait)
};

cudaError_t launch_step(const StepLaunch& a);
// the 3D step's z-chunk length and count for this problem (requested <= 0: automatic)
template <typename T>
cudaError_t step3d_chunks(const HostProblem& P, int requested, int* zchunk, int* nchunks);
size_t step_smem_bytes(int precision, int dim);

// Diagnostics.  `scratch` must hold diag_scratch_doubles(prob) doubles
// (2 DIAG_MAX_BLOCKS: one partial pair per block of a reduction grid of at most
// 8 blocks per SM and at most DIAG_MAX_BLOCKS blocks); results are written as
// doubles to out (device pointer):
//   energy_solute: out[0] = F_h, out[1] = S_h
//   front:         out[0] = x_front (local, without the window offset; NaN if
//                  none), out[1] = c_max
constexpr int DIAG_MAX_BLOCKS = 2048;
size_t diag_scratch_doubles(const HostProblem& P);
cudaError_t launch_energy_solute(const HostProblem& P, const Fields& f, int64_t step,
                                 int64_t shifts, bool with_energy, double* scratch, double* out,
                                 cudaStream_t s, long long* slot = nullptr);
cudaError_t launch_front(const HostProblem& P, const Fields& f, double* scratch, double* out,
                         cudaStream_t s);
// energy_solute (with energy) from the caller's fields (phi, c_s, c_l) of P's
// precision instead of a handle's state; same kernel, same reduction grid
cudaError_t launch_energy_solute_fields(const HostProblem& P, const void* phi, const void* cs, const void* cl,
                                        int64_t step, int64_t shifts, double* scratch, double* out,
                                        cudaStream_t s);
// moving window: out[i] = in[i+1] (i < n-1), out[n-1] = the Dirichlet state (1D)
cudaError_t launch_shift(const HostProblem& P, const Fields& in, const Fields& out, cudaStream_t s);
// (phi, c_s, c_l) of the caller's precision <-> the device state (phi, c, d[, c_lo])
cudaError_t launch_to_state(const HostProblem& P, const void* phi, const void* cs, const void* cl,
                            const Fields& out, cudaStream_t s);
// the same for cells [first, first + count) only, on `blocks` blocks (<= 0: as
// launch_to_state): one z-slab of a 3D grid, converted while earlier slabs step
cudaError_t launch_to_state_range(const HostProblem& P, const void* phi, const void* cs, const void* cl,
                                  const Fields& out, long long first, long long count, int blocks,
                                  cudaStream_t s);
void set_create_error(const std::string& msg);

// One-time set-up of a kernel's launch attributes, per device: function
// attributes such as the dynamic shared-memory limit belong to the device the
// kernel is configured on, so a process that uses several GPUs configures each.
struct DeviceSetup {
    static constexpr int MAX_DEVICES = 64;
    std::mutex mu;
    bool done[MAX_DEVICES] = {};
    int per_sm[MAX_DEVICES] = {};
    int sms[MAX_DEVICES] = {};
    size_t value[MAX_DEVICES] = {};
    cudaError_t err[MAX_DEVICES] = {};
};

// state -> (phi, c_s, c_l); blocks <= 0: the reductions' grid, else that many
// blocks (a read-back that shares the SMs and the host link with an upload)
cudaError_t launch_from_state(const HostProblem& P, const Fields& in, void* phi, void* cs, void* cl,
                              cudaStream_t s, int blocks = 0);

// The checks of pf_create on a problem description (pf_api.cu): "" if valid,
// else the reason.  stepping = false leaves out what only the time step needs
// (the explicit stability bound on dt, the moving window, the launch limits of
// the 2D/3D step kernels) and requires dt to be finite only.
std::string validate_problem(const pf_grid* grid, const pf_bc* bc, const pf_params* params, bool stepping);
// HostProblem from a validated description
void fill_problem(HostProblem& P, const pf_grid* grid, const pf_bc* bc, const pf_params* params);

}  // namespace pf
