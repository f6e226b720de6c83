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
// device array instead of a cudaMalloc'd buffer.  The reduction itself is the
// one pf_energy runs (launch_energy_solute_fields in pf_diag.cu): the same
// kernel, the same grid, only the scratch differs.
//
// The scratch array is shared by every call in the process (and stays resident
// on every GPU that loads the library until exit).  Each call overwrites all
// the partials it later reads, so nothing has to be cleared between calls, but
// two calls whose kernels overlap on the GPU (different streams, no ordering)
// race on it and may return wrong results: serialise them.
#include <cstdint>
#include <string>
#include "pf.h"
#include "pf_internal.cuh"
#include "pf_kernels.h"

namespace pf {

static constexpr long long NOALLOC_MAX_CELLS = 1LL << 30;    // largest grid accepted

// block partials of the two sums: 2 x DIAG_MAX_BLOCKS doubles = 32 KiB
static __device__ __align__(256) double g_noalloc_scratch[2 * DIAG_MAX_BLOCKS];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// on every call (cheap, allocates nothing); the first lookup on a device loads
// the library's device code there.
static double* scratch_address(cudaError_t* err) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    return *err == cudaSuccess ? static_cast<double*>(p) : nullptr;
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
    // the checks of pf_create, without those only the time step needs
    const std::string why = validate_problem(grid, bc, params, false);
    if (!why.empty()) {
        set_create_error("pf_energy_solute_noalloc: " + why);
        return PF_EINVAL;
    }
    if (step < 0 || shifts < 0) {
        set_create_error("pf_energy_solute_noalloc: negative clock");
        return PF_EINVAL;
    }
    const long long cells = grid->n[0] * grid->n[1] * grid->n[2];
    if (cells > NOALLOC_MAX_CELLS) {
        set_create_error("pf_energy_solute_noalloc: grid exceeds the 2^30-cell maximum");
        return PF_EINVAL;
    }
    cudaError_t e = cudaSuccess;
    double* part = scratch_address(&e);
    if (e != cudaSuccess || !part) {
        cudaGetLastError();
        set_create_error(std::string("pf_energy_solute_noalloc: scratch set-up: ") + cudaGetErrorString(e));
        return PF_ECUDA;
    }
    HostProblem P;
    fill_problem(P, grid, bc, params);
    e = launch_energy_solute_fields(P, phi, cs, cl, step, shifts, part, out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        set_create_error(std::string("pf_energy_solute_noalloc: launch: ") + cudaGetErrorString(e));
        return PF_ECUDA;
    }
    return PF_OK;
}
