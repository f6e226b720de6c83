// pf_api.cu -- the extern "C" boundary of libpf (declared in include/pf.h):
// validation, device state, stream-ordered stepping and diagnostics.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include "pf.h"
#include "pf_kernels.h"

struct pf_handle {
    pf::HostProblem P;
    cudaStream_t stream = nullptr;
    pf::Fields buf[2] = {{nullptr, nullptr, nullptr, nullptr, nullptr},
                         {nullptr, nullptr, nullptr, nullptr, nullptr}};
    int cur = 0;
    int64_t step = 0, shifts = 0;
    double* scratch = nullptr;   // diagnostics partials
    double* dres = nullptr;      // device results (4 doubles), then the step kernels' error flag
    double* hres = nullptr;      // pinned host results (4 doubles), then the flag's copy
    int* derr = nullptr;         // the flag: a bounded wait in a step kernel ran out
    double* drec = nullptr;      // per-step (F_h, S_h) records of pf_step_energies
    int64_t rec_cap = 0;
    // pf_set_fields_step: a conversion stream, chunk streams, one event per slab
    static constexpr int OV_STREAMS = 4;
    cudaStream_t ov[OV_STREAMS] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> ov_ev;
    // z-slab of a decomposed grid: which z sides are halo sides, whether each
    // has been imported for the current state, and the padded allocations
    // (two ghost planes below and above; buf[b] points at plane 0 of them)
    bool halo[2] = {false, false};
    bool halo_set[2] = {false, false};
    void* alloc[2][5] = {{nullptr, nullptr, nullptr, nullptr, nullptr},
                         {nullptr, nullptr, nullptr, nullptr, nullptr}};
    // pf_get_fields_async: a read-back stream, an event recorded on the handle's
    // stream before it and one after the read-back; pending while no later work
    // of the handle has been ordered after it
    cudaStream_t rb = nullptr;
    // device staging of the converted fields, two sets used in turn, so that a
    // read-back's conversion need not wait for the previous one's host copies;
    // the conversions run on rb_cv, the copies on rb
    void* rb_stage[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    int rb_slot = 0;
    cudaStream_t rb_cv = nullptr;
    cudaEvent_t rb_copied[2] = {nullptr, nullptr};   // the host copies out of staging set s are done
    bool rb_copy = true;         // read-backs to host: staged + copy engine (true) or kernel-written
    // pf_set_fields_step from page-locked host memory: slabs copied by the copy
    // engine into a device staging buffer (on their own stream, one event per
    // slab) and converted from there; up_kernel = the conversion reads the host
    // memory itself instead
    void* up_stage[3] = {nullptr, nullptr, nullptr};
    cudaStream_t up_cp = nullptr;
    std::vector<cudaEvent_t> cp_ev;
    bool up_kernel = false;
    cudaEvent_t rb_start = nullptr, rb_done = nullptr;
    cudaEvent_t rb_read = nullptr;   // the read-back has read the state (before its host copies)
    bool rb_pending = false;
    int zchunk = 0;              // z planes per CTA (3D); 0 = automatic
    int ovchunk = 16;            // z planes per slab and CTA in pf_set_fields_step
    bool generic = false;        // run 2D / 3D through the generic kernel (cross-check)
    bool no_tma = false;         // 3D: per-cell plane copies instead of TMA boxes (cross-check)
    bool drop_copies = false;    // 3D TMA: copies left out, to test the bounded wait
    bool have_front = false;
    double last_xf = 0.0, last_t = 0.0;
    // pf_step_begin / pf_step_end: the interior chunks' stream, the event it
    // waits on (recorded on the handle's stream) and the one it records; split
    // = a step is open, its interior being chunks [split_lo, split_hi)
    cudaStream_t sp = nullptr;
    cudaEvent_t sp_start = nullptr, sp_done = nullptr;
    bool split = false;
    int split_lo = 0, split_hi = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

// Page-locked host memory is readable by a kernel itself (over NVLink-C2C or
// PCIe): replace the three host pointers by their device views if all three
// are page-locked; false (pointers unchanged) otherwise.
bool device_views(const void* src[3]) {
    const void* v[3];
    for (int f = 0; f < 3; ++f) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, src[f]) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) return false;
        v[f] = at.devicePointer;
    }
    for (int f = 0; f < 3; ++f) src[f] = v[f];
    return true;
}

int fail(pf_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(pf_handle* h, cudaError_t e, const char* what) {
    return fail(h, PF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// PF_EINVAL while a split step (pf_step_begin) is open: for the calls that
// change the state or the clock
int split_closed(pf_handle* h) {
    if (h->split) return fail(h, PF_EINVAL, "a split step is open: pf_step_end first");
    return PF_OK;
}

// one step from `in` to `out` on stream s, the handle's options; all z-chunks
pf::StepLaunch step_launch(pf_handle* h, const pf::Fields& in, const pf::Fields& out, cudaStream_t s) {
    pf::StepLaunch a;
    a.prob = &h->P;
    a.phi_in = in.phi; a.c_in = in.c; a.d_in = in.d; a.clo_in = in.clo; a.plo_in = in.plo;
    a.phi_out = out.phi; a.c_out = out.c; a.d_out = out.d; a.clo_out = out.clo; a.plo_out = out.plo;
    a.step = h->step;
    a.shifts = h->shifts;
    a.zchunk = h->zchunk;
    a.use_generic = h->generic;
    a.stream = s;
    a.err = h->derr;
    a.no_tma = h->no_tma;
    a.drop_copies = h->drop_copies;
    return a;
}

// order the handle's stream after the state read of a pending
// pf_get_fields_async (before any work that may overwrite that state; its
// copies to the host may still run)
int join_readback(pf_handle* h) {
    if (!h->rb_pending) return PF_OK;
    cudaError_t e = cudaStreamWaitEvent(h->stream, h->rb_read, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "read-back join");
    h->rb_pending = false;
    return PF_OK;
}

double effective_dmax(const pf_params* p) {
    const double cs = p->k_e * p->c_inf, cl = p->c_inf;
    const double Ms = (p->mobility_mode == PF_MOBILITY_CONST) ? p->D_s : p->D_s * cs;
    const double Ml = (p->mobility_mode == PF_MOBILITY_CONST) ? p->D_l : p->D_l * cl;
    double dmax = std::fmax(Ms / cs, Ml / cl);
    const int S = 2001;
    for (int i = 0; i < S; ++i) {
        const double pp = (double)i / (S - 1);
        const double Mbar = Ms * (1.0 - pp) + p->b * Ml * pp;
        const double q = Ms * Ml * (p->b * pp + 1.0 - pp) / Mbar;
        dmax = std::fmax(dmax, q * (pp / cs + (1.0 - pp) / cl));
    }
    return dmax;
}

double stable_dt(const pf_grid* g, const pf_params* p) {
    const double lam = 4.0 * g->dim / (g->dx * g->dx);
    const double dt_phi = 2.0 / (p->M_phi * (lam * p->sigma + 2.0 * p->H));
    const double dt_c = 2.0 / (lam * effective_dmax(p));
    return std::fmin(dt_phi, dt_c);
}

// the step kernels' error flag, copied to hres[4] on the handle's stream by
// the caller's copy: PF_ETIMEOUT (and the flag cleared) if it was set
int step_error(pf_handle* h) {
    if (*reinterpret_cast<const int*>(h->hres + 4) == 0) return PF_OK;
    *reinterpret_cast<int*>(h->hres + 4) = 0;
    cudaError_t e = cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "error flag reset");
    return fail(h, PF_ETIMEOUT, "a step kernel's bounded wait for its plane copies ran out; the state is not valid");
}

}  // namespace

namespace pf {

std::string validate_problem(const pf_grid* g, const pf_bc* bc, const pf_params* p, bool stepping) {
    if (!g || !bc || !p) return "null argument";
    if (g->dim < 1 || g->dim > 3) return "dim must be 1, 2 or 3";
    for (int a = 0; a < 3; ++a) {
        if (a < g->dim) {
            if (g->n[a] < 3) return "each active axis needs at least 3 cells";
            const int lo = bc->lo[a], hi = bc->hi[a];
            if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return "unknown boundary condition";
            if ((lo == PF_BC_HALO || hi == PF_BC_HALO) && !(stepping && g->dim == 3 && a == 2))
                return "halo sides are only for the z ends of a 3D handle";
            if ((lo == PF_BC_PERIODIC) != (hi == PF_BC_PERIODIC))
                return "periodic boundaries must be set on both sides of an axis";
        } else if (g->n[a] != 1) {
            return "inactive axes must have n = 1";
        }
    }
    if (g->n[0] > (1 << 30) || g->n[1] > (1 << 30) || g->n[2] > (1 << 30) ||
        g->n[0] * g->n[1] * g->n[2] > (int64_t(1) << 34))
        return "grid too large";
    // launch limits of the 2D/3D kernels: one CTA row per 8 or 16 cells of y in
    // grid.y (at most 65535), and 32-bit offsets within an x-y plane
    if (stepping && g->dim >= 2 && g->n[1] > int64_t(65535) * 8) return "n[1] above 524280 is not supported";
    if (stepping && g->dim == 3 && g->n[0] * g->n[1] > int64_t(0x7fffffff))
        return "an x-y plane above 2^31 - 1 cells is not supported";
    if (!(g->dx > 0) || !std::isfinite(g->dx)) return "dx must be positive and finite";
    if (p->precision != PF_FP32 && p->precision != PF_FP64) return "precision must be PF_FP32 or PF_FP64";
    if (p->interp != PF_INTERP_QUINTIC && p->interp != PF_INTERP_CUBIC) return "unknown interp";
    if (p->mobility_mode != PF_MOBILITY_DC && p->mobility_mode != PF_MOBILITY_CONST)
        return "unknown mobility_mode";
    const int L = p->lap_stencil;
    if ((g->dim == 1 && L != 3) || (g->dim == 2 && L != 5 && L != 9) ||
        (g->dim == 3 && L != 7 && L != 19))
        return "lap_stencil must be 3 (1D), 5/9 (2D) or 7/19 (3D)";
    if (!(p->H > 0) || !(p->sigma > 0) || !(p->M_phi > 0) || !(p->D_s > 0) || !(p->D_l > 0))
        return "H, sigma, M_phi, D_s and D_l must be positive";
    if (!(p->k_e > 0 && p->k_e < 1)) return "k_e must lie in (0, 1)";
    if (!(p->b > 0)) return "b must be positive";
    if (!(p->delta >= 0)) return "delta must be non-negative";
    if (!(p->c_inf > 0)) return "c_inf must be positive";
    if (!std::isfinite(p->H) || !std::isfinite(p->sigma) || !std::isfinite(p->M_phi) || !std::isfinite(p->D_s) ||
        !std::isfinite(p->D_l) || !std::isfinite(p->b) || !std::isfinite(p->delta) || !std::isfinite(p->c_inf) ||
        !std::isfinite(p->A) || !std::isfinite(p->a) || !std::isfinite(p->theta_ref) ||
        !std::isfinite(p->G_theta) || !std::isfinite(p->v_pull) || !std::isfinite(p->x0) ||
        !std::isfinite(bc->dir_phi) || !std::isfinite(bc->dir_cs) || !std::isfinite(bc->dir_cl))
        return "non-finite parameter";
    if (!stepping) return std::isfinite(p->dt) ? "" : "non-finite parameter";
    if (p->shift && g->dim != 1) return "the moving window is supported in 1D only";
    if (p->shift && !(p->v_pull * p->dt < g->dx)) return "v_pull dt must be below dx";
    if (!(p->dt > 0)) return "dt must be positive";
    const double dts = stable_dt(g, p);
    if (p->dt > dts * (1.0 + 1e-12)) return "dt exceeds the explicit stability bound";
    return "";
}

void fill_problem(HostProblem& P, const pf_grid* grid, const pf_bc* bc, const pf_params* params) {
    P.dim = grid->dim;
    for (int a = 0; a < 3; ++a) {
        P.n[a] = (a < grid->dim) ? grid->n[a] : 1;
        P.bc_lo[a] = (a < grid->dim) ? bc->lo[a] : PF_BC_NOFLUX;
        P.bc_hi[a] = (a < grid->dim) ? bc->hi[a] : PF_BC_NOFLUX;
    }
    P.dx = grid->dx;
    P.dir_phi = bc->dir_phi; P.dir_cs = bc->dir_cs; P.dir_cl = bc->dir_cl;
    P.precision = params->precision;
    P.interp = params->interp;
    P.lap = params->lap_stencil;
    P.mobility = params->mobility_mode;
    P.H = params->H; P.sigma = params->sigma; P.M_phi = params->M_phi;
    P.D_s = params->D_s; P.D_l = params->D_l; P.k_e = params->k_e;
    P.A = params->A; P.b = params->b; P.a = params->a; P.delta = params->delta;
    P.theta_ref = params->theta_ref; P.G_theta = params->G_theta;
    P.v_pull = params->v_pull; P.x0 = params->x0; P.dt = params->dt; P.c_inf = params->c_inf;
    P.shift = params->shift ? 1 : 0;
}

}  // namespace pf

namespace pf {
// message returned by pf_last_error(NULL) (failed pf_create / pf_run_batch)
void set_create_error(const std::string& msg) { g_create_error = msg; }
}  // namespace pf

extern "C" {

const char* pf_last_error(pf_handle* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

int pf_stable_dt(const pf_grid* grid, const pf_params* params, double* dt) {
    if (!grid || !params || !dt) return fail(nullptr, PF_EINVAL, "null argument");
    if (grid->dim < 1 || grid->dim > 3 || !(grid->dx > 0) || !(params->M_phi > 0) ||
        !(params->k_e > 0 && params->k_e < 1) || !(params->b > 0) || !(params->c_inf > 0))
        return fail(nullptr, PF_EINVAL, "invalid grid or parameters");
    *dt = stable_dt(grid, params);
    return PF_OK;
}

int pf_create(const pf_grid* grid, const pf_bc* bc, const pf_params* params, void* stream,
              pf_handle** out) {
    if (!out) return fail(nullptr, PF_EINVAL, "null output pointer");
    *out = nullptr;
    const std::string why = pf::validate_problem(grid, bc, params, true);
    if (!why.empty()) return fail(nullptr, PF_EINVAL, why);
    pf_handle* h = new (std::nothrow) pf_handle();
    if (!h) return fail(nullptr, PF_ENOMEM, "host allocation failed");
    pf::HostProblem& P = h->P;
    pf::fill_problem(P, grid, bc, params);
    h->stream = static_cast<cudaStream_t>(stream);
    if (const char* zc = std::getenv("PF_ZCHUNK")) h->zchunk = std::atoi(zc);   // tuning override
    if (const char* oc = std::getenv("PF_OVCHUNK")) h->ovchunk = std::atoi(oc);
    if (const char* g = std::getenv("PF_GENERIC")) h->generic = std::atoi(g) != 0;   // cross-check kernel
    if (const char* t = std::getenv("PF_TMA")) h->no_tma = std::atoi(t) == 0;           // cross-check staging
    if (const char* t = std::getenv("PF_TEST_DROP_COPIES")) h->drop_copies = std::atoi(t) != 0;
    if (const char* r = std::getenv("PF_READBACK")) h->rb_copy = std::strcmp(r, "direct") != 0;
    if (const char* u = std::getenv("PF_UPLOAD")) h->up_kernel = std::strcmp(u, "kernel") == 0;

    h->halo[0] = P.bc_lo[2] == PF_BC_HALO;
    h->halo[1] = P.bc_hi[2] == PF_BC_HALO;
    // a slab keeps two ghost planes below and above its own planes; the space
    // below is rounded up to 256 bytes so that plane 0 keeps cudaMalloc's
    // alignment (the FP32 solute reduction reads c and c_lo as float4)
    const size_t ghost_bytes = (h->halo[0] || h->halo[1]) ? 2 * (size_t)P.n[0] * P.n[1] * P.elem() : 0;
    const size_t lead = (ghost_bytes + 255) / 256 * 256;
    const size_t bytes = lead + (size_t)P.cells() * P.elem() + ghost_bytes;
    for (int b = 0; b < 2; ++b) {
        void** slots[5] = {&h->buf[b].phi, &h->buf[b].c, &h->buf[b].d, &h->buf[b].clo, &h->buf[b].plo};
        // FP32 keeps the low word of c, and in 1D also that of phi
        const int nf = (P.precision == PF_FP32) ? (P.dim == 1 ? 5 : 4) : 3;
        for (int f = 0; f < nf; ++f) {
            cudaError_t e = cudaMalloc(&h->alloc[b][f], bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                h->alloc[b][f] = nullptr;
                pf_destroy(h);
                return fail(nullptr, PF_ENOMEM, std::string("device allocation failed: ") +
                                                    cudaGetErrorString(e));
            }
            *slots[f] = static_cast<char*>(h->alloc[b][f]) + lead;
        }
    }
    cudaError_t e = cudaMalloc(&h->scratch, pf::diag_scratch_doubles(P) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->dres, 5 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&h->hres, 5 * sizeof(double));
    if (e == cudaSuccess) {
        h->derr = reinterpret_cast<int*>(h->dres + 4);
        e = cudaMemset(h->derr, 0, sizeof(int));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        pf_destroy(h);
        return fail(nullptr, PF_ENOMEM, std::string("allocation failed: ") + cudaGetErrorString(e));
    }
    *out = h;
    return PF_OK;
}

void pf_destroy(pf_handle* h) {
    if (!h) return;
    if (h->sp) cudaStreamSynchronize(h->sp);
    if (h->rb_cv) cudaStreamSynchronize(h->rb_cv);
    if (h->rb) cudaStreamSynchronize(h->rb);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->sp) cudaStreamDestroy(h->sp);
    if (h->sp_start) cudaEventDestroy(h->sp_start);
    if (h->sp_done) cudaEventDestroy(h->sp_done);
    if (h->rb) cudaStreamDestroy(h->rb);
    if (h->rb_cv) cudaStreamDestroy(h->rb_cv);
    if (h->rb_start) cudaEventDestroy(h->rb_start);
    if (h->rb_done) cudaEventDestroy(h->rb_done);
    if (h->rb_read) cudaEventDestroy(h->rb_read);
    for (cudaEvent_t ev : h->rb_copied)
        if (ev) cudaEventDestroy(ev);
    for (auto& set : h->rb_stage)
        for (void* p : set)
            if (p) cudaFree(p);
    for (void* p : h->up_stage)
        if (p) cudaFree(p);
    if (h->up_cp) cudaStreamDestroy(h->up_cp);
    for (cudaEvent_t ev : h->cp_ev) cudaEventDestroy(ev);
    for (int b = 0; b < 2; ++b)
        for (void* p : h->alloc[b])
            if (p) cudaFree(p);
    if (h->scratch) cudaFree(h->scratch);
    if (h->dres) cudaFree(h->dres);
    if (h->hres) cudaFreeHost(h->hres);
    if (h->drec) cudaFree(h->drec);
    for (cudaStream_t s : h->ov)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t ev : h->ov_ev) cudaEventDestroy(ev);
    delete h;
}

int pf_set_fields(pf_handle* h, const void* phi, const void* cs, const void* cl, int where) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (int rc = split_closed(h)) return rc;
    if (!phi || !cs || !cl) return fail(h, PF_EINVAL, "null field pointer");
    if (where != PF_HOST && where != PF_DEVICE) return fail(h, PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    if (int rc = join_readback(h)) return rc;
    const size_t bytes = (size_t)h->P.cells() * h->P.elem();
    const void* src[3] = {phi, cs, cl};
    const bool mapped = where == PF_HOST && device_views(src);
    if (where == PF_HOST && !mapped) {
        // stage (phi, c_s, c_l) in the idle ping-pong buffer, then convert
        const pf::Fields& st = h->buf[h->cur ^ 1];
        void* dst[3] = {st.phi, st.c, st.d};
        for (int f = 0; f < 3; ++f) {
            cudaError_t e = cudaMemcpyAsync(dst[f], src[f], bytes, cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync");
        }
        for (int f = 0; f < 3; ++f) src[f] = dst[f];
    }
    cudaError_t e = pf::launch_to_state(h->P, src[0], src[1], src[2], h->buf[h->cur], h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "state conversion");
    h->have_front = false;
    h->halo_set[0] = h->halo_set[1] = false;
    if (where == PF_HOST) {
        // the caller may reuse its host memory as soon as we return
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    }
    return PF_OK;
}

int pf_set_fields_step(pf_handle* h, const void* phi, const void* cs, const void* cl, int where,
                       int64_t n) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (int rc = split_closed(h)) return rc;
    if (!phi || !cs || !cl) return fail(h, PF_EINVAL, "null field pointer");
    if (where != PF_HOST && where != PF_DEVICE && where != PF_HOST_ASYNC)
        return fail(h, PF_EINVAL, "where must be PF_HOST, PF_HOST_ASYNC or PF_DEVICE");
    if (n < 0) return fail(h, PF_EINVAL, "negative step count");
    if (h->halo[0] || h->halo[1])
        return fail(h, PF_EINVAL, "a slab with halo sides sets its fields, imports its halos, then steps");
    // PF_HOST_ASYNC: page-locked host memory, the host not waiting for its copies
    const bool no_wait = where == PF_HOST_ASYNC;
    if (no_wait) where = PF_HOST;
    const pf::HostProblem& P = h->P;
    const void* src[3] = {phi, cs, cl};
    const void* host[3] = {phi, cs, cl};
    const bool readable = where == PF_DEVICE || device_views(src);
    if (no_wait && !readable) return fail(h, PF_EINVAL, "PF_HOST_ASYNC needs page-locked host memory");
    int zchunk = 0, nch = 0;
    cudaError_t e = cudaSuccess;
    if (P.dim == 3 && !h->generic && n > 0 && readable) {
        // Short slabs: the last chunk of the first step, which can only start
        // once the whole state is in, is then short too.  The extra halo planes
        // they cost are computed while the SMs would otherwise wait on the link.
        int req = h->ovchunk > 0 ? h->ovchunk : 16;
        if (h->zchunk > 0) req = std::min(req, h->zchunk);
        e = P.precision == 1 ? pf::step3d_chunks<double>(P, req, &zchunk, &nch)
                             : pf::step3d_chunks<float>(P, req, &zchunk, &nch);
        if (e != cudaSuccess) return cuda_fail(h, e, "step setup");
    }
    if (nch < 2) {   // nothing to overlap: the two calls in sequence
        int rc = pf_set_fields(h, phi, cs, cl, where);
        return rc ? rc : pf_step(h, n);
    }
    // streams and per-slab events, made once per handle
    for (int i = 0; i < pf_handle::OV_STREAMS && e == cudaSuccess; ++i) {
        if (h->ov[i]) continue;
        int lo = 0, hi = 0;
        if (i == 0) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);   // conversion first
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->ov[i], cudaStreamNonBlocking, i == 0 ? hi : lo);
    }
    while (e == cudaSuccess && (int)h->ov_ev.size() < nch + 1) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) h->ov_ev.push_back(ev);
    }
    // host slabs through the copy engine: a kernel reading page-locked memory
    // and a copy engine writing it (a pending read-back) do not share the host
    // link as two copy engines do (measured on a 256^3 state: device-to-host
    // and host-to-device copies side by side in 1.23 ms against 1.05 + 0.96 ms
    // one after the other)
    const bool ce = where == PF_HOST && !h->up_kernel;
    const size_t elem = P.elem();
    if (ce && e == cudaSuccess) {
        for (int f = 0; f < 3 && e == cudaSuccess; ++f)
            if (!h->up_stage[f]) {
                e = cudaMalloc(&h->up_stage[f], (size_t)P.cells() * elem);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    h->up_stage[f] = nullptr;
                    return fail(h, PF_ENOMEM, std::string("upload staging: ") + cudaGetErrorString(e));
                }
            }
        if (!h->up_cp) e = cudaStreamCreateWithFlags(&h->up_cp, cudaStreamNonBlocking);
        while (e == cudaSuccess && (int)h->cp_ev.size() < nch) {
            cudaEvent_t ev = nullptr;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) h->cp_ev.push_back(ev);
        }
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "stream setup");
    cudaStream_t conv = h->ov[0];
    cudaEvent_t start = h->ov_ev[nch];
    // The upload is converted into the idle state buffer (the input of the
    // handle's last step, free once the work queued on its stream is done) and
    // the step writes the current one.  A pending pf_get_fields_async reads the
    // current buffer, so the upload overlaps that read-back; only the step
    // chunks wait for it.
    const int src_buf = h->cur ^ 1, dst_buf = h->cur;
    // Slab j (the planes of z-chunk j) is converted on `conv` after the work
    // already queued on the handle's stream; chunk j of the first step starts
    // once every plane it reads (z0 - 2 .. z1 + 1, wrapped on a periodic z
    // axis) has been converted, on one of the chunk streams, so that the step
    // of the first slabs runs while the later ones are still being read.
    const long long plane = P.n[0] * P.n[1];
    const int nz = (int)P.n[2];
    int dev = 0, nsms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "device query");
    if (e == cudaSuccess) e = cudaEventRecord(start, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(conv, start, 0);
    for (int j = 0; j < nch && e == cudaSuccess; ++j) {
        const long long z0 = (long long)j * zchunk, z1 = std::min<long long>(nz, z0 + zchunk);
        const void* from[3] = {src[0], src[1], src[2]};
        if (ce) {
            // the slab's three fields by the copy engine, then converted from
            // device memory once they are in
            const size_t off = (size_t)(z0 * plane) * elem, len = (size_t)((z1 - z0) * plane) * elem;
            // the staging slab is free once the previous call's conversion of
            // it is done (its event, not yet re-recorded by this call); the
            // copies need not wait for the previous step, which the
            // conversion below does wait for
            e = cudaStreamWaitEvent(h->up_cp, h->ov_ev[j], 0);
            for (int f = 0; f < 3 && e == cudaSuccess; ++f)
                e = cudaMemcpyAsync(static_cast<char*>(h->up_stage[f]) + off, static_cast<const char*>(host[f]) + off,
                                    len, cudaMemcpyHostToDevice, h->up_cp);
            if (e == cudaSuccess) e = cudaEventRecord(h->cp_ev[j], h->up_cp);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(conv, h->cp_ev[j], 0);
            for (int f = 0; f < 3; ++f) from[f] = h->up_stage[f];
        }
        // two blocks per SM: the conversion is bound by the host link (or, from
        // the staging buffer, brief), and leaves the SMs to the step chunks
        if (e == cudaSuccess)
            e = pf::launch_to_state_range(P, from[0], from[1], from[2], h->buf[src_buf], z0 * plane,
                                          (z1 - z0) * plane, 2 * nsms, conv);
        if (e == cudaSuccess) e = cudaEventRecord(h->ov_ev[j], conv);
    }
    const pf::Fields& in = h->buf[src_buf];
    const pf::Fields& out = h->buf[dst_buf];
    const bool zper = P.bc_lo[2] == PF_BC_PERIODIC;
    for (int i = 1; i < pf_handle::OV_STREAMS && e == cudaSuccess && h->rb_pending; ++i)
        e = cudaStreamWaitEvent(h->ov[i], h->rb_read, 0);
    for (int j = 0; j < nch && e == cudaSuccess; ++j) {
        const int z0 = j * zchunk, z1 = std::min(nz, z0 + zchunk);
        int need = std::min(nch - 1, std::min(nz - 1, z1 + 1) / zchunk);
        if (zper && (z0 - 2 < 0 || z1 + 1 >= nz)) need = nch - 1;
        // three chunk streams: a chunk has one CTA per SM, so several run side by
        // side (measured: 1.46 ms per call with one stream, 1.18 with two, 1.13 with three)
        cudaStream_t ks = h->ov[1 + j % (pf_handle::OV_STREAMS - 1)];
        e = cudaStreamWaitEvent(ks, h->ov_ev[need], 0);
        if (e != cudaSuccess) break;
        pf::StepLaunch a;
        a.prob = &P;
        a.phi_in = in.phi; a.c_in = in.c; a.d_in = in.d; a.clo_in = in.clo; a.plo_in = in.plo;
        a.phi_out = out.phi; a.c_out = out.c; a.d_out = out.d; a.clo_out = out.clo; a.plo_out = out.plo;
        a.step = h->step;
        a.shifts = h->shifts;
        a.zchunk = zchunk;
        a.zfirst = j;
        a.zcount = 1;
        a.use_generic = false;
        a.stream = ks;
        a.err = h->derr;
        a.no_tma = h->no_tma;
        a.drop_copies = h->drop_copies;
        e = pf::launch_step(a);
    }
    // the handle's stream continues after every chunk
    for (int i = 1; i < pf_handle::OV_STREAMS && e == cudaSuccess; ++i) {
        e = cudaEventRecord(start, h->ov[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, start, 0);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "overlapped upload and step");
    h->rb_pending = false;   // the handle's stream now follows the read-back too
    h->have_front = false;
    h->step += 1;
    if (where == PF_HOST && !no_wait) {
        // the caller may reuse its host memory once the last slab is read
        e = cudaEventSynchronize(ce ? h->cp_ev[nch - 1] : h->ov_ev[nch - 1]);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
    }
    return pf_step(h, n - 1);
}

int pf_get_fields_async(pf_handle* h, void* phi, void* cs, void* cl, int where) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (!phi || !cs || !cl) return fail(h, PF_EINVAL, "null field pointer");
    if (where != PF_HOST && where != PF_DEVICE) return fail(h, PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    void* tgt[3] = {phi, cs, cl};
    const size_t bytes = (size_t)h->P.cells() * h->P.elem();
    if (where == PF_HOST) {
        const void* views[3] = {phi, cs, cl};
        if (!device_views(views)) return fail(h, PF_EINVAL, "pf_get_fields_async needs page-locked host memory");
        for (int f = 0; f < 3; ++f) tgt[f] = const_cast<void*>(views[f]);
    }
    // host outputs converted into a staging set of the handle's own (the
    // idle state buffer is the next upload's target), then copied by the copy
    // engine (PF_READBACK=direct: written by the conversion kernel itself)
    const bool staged = where == PF_HOST && h->rb_copy;
    const int slot = h->rb_slot;
    if (staged) {
        for (int f = 0; f < 3; ++f) {
            if (!h->rb_stage[slot][f]) {
                cudaError_t a = cudaMalloc(&h->rb_stage[slot][f], bytes);
                if (a != cudaSuccess) {
                    cudaGetLastError();
                    h->rb_stage[slot][f] = nullptr;
                    return fail(h, PF_ENOMEM, std::string("read-back staging: ") + cudaGetErrorString(a));
                }
            }
            tgt[f] = h->rb_stage[slot][f];
        }
    }
    cudaError_t e = cudaSuccess;
    if (!h->rb) {
        e = cudaStreamCreateWithFlags(&h->rb, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->rb_cv, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->rb_start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->rb_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->rb_read, cudaEventDisableTiming);
        for (int s2 = 0; s2 < 2 && e == cudaSuccess; ++s2)
            e = cudaEventCreateWithFlags(&h->rb_copied[s2], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(h, e, "read-back stream");
    }
    // written by the kernel: two blocks per SM (bound by the link or DRAM, the
    // SMs left to an upload's conversion and steps); staged: the conversion
    // on the full grid, then the copy engine.  The conversion (rb_cv) waits for
    // the work queued on the handle's stream and, staged, for the host copies
    // that last read its staging set; the copies (rb) follow the conversion.
    int dev = 0, nsms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaEventRecord(h->rb_start, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->rb_cv, h->rb_start, 0);
    if (e == cudaSuccess && staged) e = cudaStreamWaitEvent(h->rb_cv, h->rb_copied[slot], 0);
    if (e == cudaSuccess)
        e = pf::launch_from_state(h->P, h->buf[h->cur], tgt[0], tgt[1], tgt[2], h->rb_cv, staged ? 0 : 2 * nsms);
    if (e == cudaSuccess) e = cudaEventRecord(h->rb_read, h->rb_cv);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->rb, h->rb_read, 0);
    void* out[3] = {phi, cs, cl};
    for (int f = 0; f < 3 && e == cudaSuccess && staged; ++f)
        e = cudaMemcpyAsync(out[f], tgt[f], bytes, cudaMemcpyDeviceToHost, h->rb);
    if (e == cudaSuccess && staged) e = cudaEventRecord(h->rb_copied[slot], h->rb);
    if (e == cudaSuccess) e = cudaEventRecord(h->rb_done, h->rb);
    if (e != cudaSuccess) return cuda_fail(h, e, "read-back");
    if (staged) h->rb_slot ^= 1;
    h->rb_pending = true;
    return PF_OK;
}

int pf_sync(pf_handle* h) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (int rc = join_readback(h)) return rc;
    cudaError_t e = cudaSuccess;
    if (h->rb) e = cudaStreamWaitEvent(h->stream, h->rb_done, 0);   // the copies to the host too
    if (e == cudaSuccess && h->split && h->split_hi > h->split_lo)
        e = cudaStreamWaitEvent(h->stream, h->sp_done, 0);          // an open split step's interior
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->hres + 4, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    return step_error(h);
}

int pf_get_fields(pf_handle* h, void* phi, void* cs, void* cl, int where) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (!phi || !cs || !cl) return fail(h, PF_EINVAL, "null field pointer");
    if (where != PF_HOST && where != PF_DEVICE) return fail(h, PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    const size_t bytes = (size_t)h->P.cells() * h->P.elem();
    void* out[3] = {phi, cs, cl};
    const pf::Fields& st = h->buf[h->cur ^ 1];
    void* tgt[3] = {phi, cs, cl};
    // host memory through a device staging copy (the idle state buffer) and the
    // copy engine (PF_READBACK=direct: page-locked memory written by the
    // conversion kernel itself, at about half the device-to-host rate)
    const void* views[3] = {phi, cs, cl};
    const bool mapped = where == PF_HOST && !h->rb_copy && device_views(views);
    if (mapped) {
        for (int f = 0; f < 3; ++f) tgt[f] = const_cast<void*>(views[f]);
    } else if (where == PF_HOST) {
        tgt[0] = st.phi; tgt[1] = st.c; tgt[2] = st.d;
    }
    cudaError_t e = pf::launch_from_state(h->P, h->buf[h->cur], tgt[0], tgt[1], tgt[2], h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "state conversion");
    if (where == PF_HOST && !mapped) {
        for (int f = 0; f < 3; ++f) {
            e = cudaMemcpyAsync(out[f], tgt[f], bytes, cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync");
        }
    }
    e = cudaMemcpyAsync(h->hres + 4, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    return step_error(h);
}

int pf_step(pf_handle* h, int64_t n) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (int rc = split_closed(h)) return rc;
    if (n < 0) return fail(h, PF_EINVAL, "negative step count");
    if (h->halo[0] || h->halo[1]) {
        if (n > 1) return fail(h, PF_EINVAL, "a slab with halo sides steps one step at a time");
        if (n == 1 && ((h->halo[0] && !h->halo_set[0]) || (h->halo[1] && !h->halo_set[1])))
            return fail(h, PF_EINVAL, "halo not imported since the last step or pf_set_fields");
        h->halo_set[0] = h->halo_set[1] = false;
    }
    if (n > 0)
        if (int rc = join_readback(h)) return rc;
    const pf::HostProblem& P = h->P;
    for (int64_t s = 0; s < n; ++s) {
        const pf::StepLaunch a = step_launch(h, h->buf[h->cur], h->buf[h->cur ^ 1], h->stream);
        cudaError_t e = pf::launch_step(a);
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel launch");
        h->cur ^= 1;
        h->step += 1;
        if (P.shift) {
            const double t = (double)h->step * P.dt;
            while (P.v_pull * t >= (double)(h->shifts + 1) * P.dx) {
                e = pf::launch_shift(P, h->buf[h->cur], h->buf[h->cur ^ 1], h->stream);
                if (e != cudaSuccess) return cuda_fail(h, e, "shift kernel launch");
                h->cur ^= 1;
                h->shifts += 1;
            }
        }
    }
    return PF_OK;
}

static int fetch_results(pf_handle* h, int count) {
    (void)count;   // the results and the error flag, in one copy
    cudaError_t e = cudaMemcpyAsync(h->hres, h->dres, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "result copy");
    return step_error(h);
}

static int energy_solute(pf_handle* h, bool with_energy) {
    cudaError_t e = pf::launch_energy_solute(h->P, h->buf[h->cur], h->step, h->shifts, with_energy,
                                             h->scratch, h->dres, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "energy kernel launch");
    return fetch_results(h, 2);
}

int pf_energy(pf_handle* h, double* F) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (!F) return fail(h, PF_EINVAL, "null output");
    if ((h->halo[0] && !h->halo_set[0]) || (h->halo[1] && !h->halo_set[1]))
        return fail(h, PF_EINVAL, "halo not imported: the energy's gradient pairs reach the ghost planes");
    int rc = energy_solute(h, true);
    if (rc) return rc;
    *F = h->hres[0];
    if (!std::isfinite(*F)) return fail(h, PF_ENONFINITE, "non-finite free energy");
    return PF_OK;
}

int pf_step_energies(pf_handle* h, int64_t n, double* F) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (int rc = split_closed(h)) return rc;
    if (n < 0) return fail(h, PF_EINVAL, "negative step count");
    if (h->halo[0] || h->halo[1]) return fail(h, PF_EINVAL, "not for a slab with halo sides");
    if (int rc = join_readback(h)) return rc;
    if (n > 0 && !F) return fail(h, PF_EINVAL, "null output");
    if (n == 0) return PF_OK;
    if (h->rec_cap < n) {
        if (h->drec) {
            cudaStreamSynchronize(h->stream);
            cudaFree(h->drec);
            h->drec = nullptr;
            h->rec_cap = 0;
        }
        // 2 n doubles of records, then the record counter
        cudaError_t e = cudaMalloc(&h->drec, 2 * (size_t)n * sizeof(double) + sizeof(long long));
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->drec = nullptr;
            return fail(h, PF_ENOMEM, std::string("record allocation failed: ") + cudaGetErrorString(e));
        }
        h->rec_cap = n;
    }
    long long* slot = reinterpret_cast<long long*>(h->drec + 2 * h->rec_cap);
    cudaError_t e = cudaMemsetAsync(slot, 0, sizeof(long long), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "record counter");
    auto one = [&]() -> int {
        int rc = pf_step(h, 1);
        if (rc) return rc;
        cudaError_t x = pf::launch_energy_solute(h->P, h->buf[h->cur], h->step, h->shifts, true, h->scratch,
                                                 h->drec, h->stream, slot);
        return x == cudaSuccess ? PF_OK : cuda_fail(h, x, "energy kernel launch");
    };
    int64_t done = 0;
    // Without a moving temperature or window every step launches the same
    // kernels with the same arguments (the ping-pong parity returns after an
    // even count, the record slot advances on the device), so a captured block
    // of GS steps is replayed instead of launching three kernels per step.
    const pf::HostProblem& P = h->P;
    constexpr int64_t GS = 64;
    if (P.G_theta == 0.0 && P.v_pull == 0.0 && !P.shift && n >= 2 + 2 * GS) {
        for (; done < 2; ++done)   // first uses set kernel attributes outside the capture
            if (int rc = one()) return rc;
        // capture and replay on a stream of our own, ordered after and before
        // the handle's stream (which may be the legacy default stream, where
        // capture is not allowed)
        cudaStream_t cap = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev, 0);
        const cudaStream_t own = h->stream;
        const int64_t step0 = h->step;
        const int cur0 = h->cur;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int rc = PF_OK;
        if (e == cudaSuccess) {
            h->stream = cap;
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            for (int64_t s = 0; s < GS && e == cudaSuccess && rc == PF_OK; ++s) rc = one();
            cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess && rc == PF_OK) e = cudaGraphInstantiate(&exec, graph, 0);
            h->step = step0;   // the capture advanced the host clock without running anything
            h->cur = cur0;
            for (; e == cudaSuccess && rc == PF_OK && n - done >= GS; done += GS) {
                e = cudaGraphLaunch(exec, cap);
                h->step += GS;
            }
            h->stream = own;
            cudaError_t e3 = cudaEventRecord(ev, cap);
            if (e3 == cudaSuccess) e3 = cudaStreamWaitEvent(own, ev, 0);
            if (e == cudaSuccess) e = e3;
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        if (ev) cudaEventDestroy(ev);
        if (rc) return rc;
        if (e != cudaSuccess) return cuda_fail(h, e, "step graph");
    }
    for (; done < n; ++done)
        if (int rc = one()) return rc;
    std::vector<double> rec(2 * (size_t)n);
    e = cudaMemcpyAsync(rec.data(), h->drec, 2 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->hres + 4, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "record copy");
    if (int rc = step_error(h)) return rc;
    bool finite = true;
    for (int64_t s = 0; s < n; ++s) {
        F[s] = rec[2 * s];
        finite = finite && std::isfinite(F[s]);
    }
    if (!finite) return fail(h, PF_ENONFINITE, "non-finite free energy");
    return PF_OK;
}

int pf_solute_total(pf_handle* h, double* S) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (!S) return fail(h, PF_EINVAL, "null output");
    int rc = energy_solute(h, false);
    if (rc) return rc;
    *S = h->hres[1];
    if (!std::isfinite(*S)) return fail(h, PF_ENONFINITE, "non-finite solute total");
    return PF_OK;
}

int pf_solute_total_async(pf_handle* h, double* S) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (!S) return fail(h, PF_EINVAL, "null output");
    cudaError_t e = pf::launch_energy_solute(h->P, h->buf[h->cur], h->step, h->shifts, false, h->scratch,
                                             h->dres, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S, h->dres + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "solute total");
    return PF_OK;
}

int pf_front(pf_handle* h, double* x_front, double* v_front, double* c_max) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (!x_front || !v_front || !c_max) return fail(h, PF_EINVAL, "null output");
    cudaError_t e = pf::launch_front(h->P, h->buf[h->cur], h->scratch, h->dres, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "front kernel launch");
    int rc = fetch_results(h, 2);
    if (rc) return rc;
    const double xf = h->hres[0] + (double)h->shifts * h->P.dx;
    const double t = (double)h->step * h->P.dt;
    *x_front = xf;
    *c_max = h->hres[1];
    *v_front = (h->have_front && t > h->last_t) ? (xf - h->last_xf) / (t - h->last_t) : NAN;
    h->have_front = true;
    h->last_xf = xf;
    h->last_t = t;
    if (!std::isfinite(*c_max)) return fail(h, PF_ENONFINITE, "non-finite concentration");
    return PF_OK;
}

// ---------------------------------------------------------------- halos

// the state words of a halo: phi, c, d and (FP32) the low word of c
static int halo_nfields(const pf_handle* h) { return h->P.precision == PF_FP32 ? 4 : 3; }

int pf_halo_bytes(pf_handle* h, int64_t* bytes) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (!bytes) return fail(h, PF_EINVAL, "null output");
    *bytes = (int64_t)halo_nfields(h) * 2 * h->P.n[0] * h->P.n[1] * (int64_t)h->P.elem();
    return PF_OK;
}

static int halo_copy(pf_handle* h, int side, void* buf, int where, bool import) {
    if (side != 0 && side != 1) return fail(h, PF_EINVAL, "side must be 0 (low z) or 1 (high z)");
    if (import)
        if (int rc = join_readback(h)) return rc;
    if (!h->halo[side]) return fail(h, PF_EINVAL, "that z side is not a halo side");
    if (!buf) return fail(h, PF_EINVAL, "null buffer");
    if (where != PF_HOST && where != PF_DEVICE) return fail(h, PF_EINVAL, "where must be PF_HOST or PF_DEVICE");
    const pf::HostProblem& P = h->P;
    const size_t plane = (size_t)P.n[0] * P.n[1] * P.elem();
    // first plane of the two: own planes 0 / nz-2 (export), ghosts -2 / nz (import)
    const int64_t z = import ? (side == 0 ? -2 : P.n[2]) : (side == 0 ? 0 : P.n[2] - 2);
    const pf::Fields& F = h->buf[h->cur];
    void* const f[4] = {F.phi, F.c, F.d, F.clo};
    const int nf = halo_nfields(h);
    const cudaMemcpyKind kind = where == PF_DEVICE ? cudaMemcpyDeviceToDevice
                                                   : (import ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
    for (int k = 0; k < nf; ++k) {
        char* state = static_cast<char*>(f[k]) + z * (int64_t)plane;
        char* ext = static_cast<char*>(buf) + (size_t)k * 2 * plane;
        cudaError_t e = import ? cudaMemcpyAsync(state, ext, 2 * plane, kind, h->stream)
                               : cudaMemcpyAsync(ext, state, 2 * plane, kind, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "halo copy");
    }
    if (where == PF_HOST) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    }
    if (import) h->halo_set[side] = true;
    return PF_OK;
}

int pf_get_halo(pf_handle* h, int side, void* buf, int where) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    return halo_copy(h, side, buf, where, false);
}

int pf_set_halo(pf_handle* h, int side, const void* buf, int where) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    return halo_copy(h, side, const_cast<void*>(buf), where, true);
}

// ---------------------------------------------------------------- split step

// The fused 3D step's z-chunk j covers planes [j zc, min(nz, (j + 1) zc)) and
// reads planes j zc - 2 .. (j + 1) zc + 1 of its input.  Chunks [*lo, *hi)
// read only planes 0 .. nz - 1 (start >= 2, end <= nz - 2): the interior,
// which needs no ghost plane.  *hi <= *lo when there is none.
static int interior_chunks(pf_handle* h, int* lo, int* hi) {
    const pf::HostProblem& P = h->P;
    int zc = 0, nch = 0;
    cudaError_t e = P.precision == 1 ? pf::step3d_chunks<double>(P, h->zchunk, &zc, &nch)
                                     : pf::step3d_chunks<float>(P, h->zchunk, &zc, &nch);
    if (e != cudaSuccess) return cuda_fail(h, e, "step setup");
    const int nz = (int)P.n[2];
    *lo = (2 + zc - 1) / zc;
    *hi = std::min(nch, std::max(0, nz - 2) / zc);
    return PF_OK;
}

int pf_step_begin(pf_handle* h) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (int rc = split_closed(h)) return rc;
    if (h->P.dim != 3 || h->generic) return fail(h, PF_EINVAL, "the split step needs a 3D grid and the fused 3D kernel");
    if (int rc = join_readback(h)) return rc;
    int lo = 0, hi = 0;
    if (int rc = interior_chunks(h, &lo, &hi)) return rc;
    cudaError_t e = cudaSuccess;
    if (!h->sp) {
        e = cudaStreamCreateWithFlags(&h->sp, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->sp_start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->sp_done, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(h, e, "split-step stream");
    }
    if (hi > lo) {
        // the interior follows everything queued on the handle's stream (the
        // previous step's last readers of the buffer it writes included)
        e = cudaEventRecord(h->sp_start, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->sp, h->sp_start, 0);
        pf::StepLaunch a = step_launch(h, h->buf[h->cur], h->buf[h->cur ^ 1], h->sp);
        a.zfirst = lo;
        a.zcount = hi - lo;
        if (e == cudaSuccess) e = pf::launch_step(a);
        if (e == cudaSuccess) e = cudaEventRecord(h->sp_done, h->sp);
        if (e != cudaSuccess) return cuda_fail(h, e, "interior step launch");
    }
    h->split = true;
    h->split_lo = lo;
    h->split_hi = hi;
    return PF_OK;
}

int pf_step_end(pf_handle* h) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (!h->split) return fail(h, PF_EINVAL, "no split step is open: pf_step_begin first");
    if ((h->halo[0] && !h->halo_set[0]) || (h->halo[1] && !h->halo_set[1]))
        return fail(h, PF_EINVAL, "halo not imported since the last step or pf_set_fields");
    if (int rc = join_readback(h)) return rc;
    const int lo = h->split_lo, hi = h->split_hi;
    h->split = false;
    pf::StepLaunch a = step_launch(h, h->buf[h->cur], h->buf[h->cur ^ 1], h->stream);
    cudaError_t e = cudaSuccess;
    if (hi > lo) {
        // the chunks below and above the interior, then the join
        a.zfirst = 0;
        a.zcount = lo;
        if (lo > 0) e = pf::launch_step(a);
        a.zfirst = hi;
        a.zcount = 1 << 30;   // to the last chunk
        if (e == cudaSuccess) e = pf::launch_step(a);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->sp_done, 0);
    } else {
        e = pf::launch_step(a);   // no interior: every chunk
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "boundary step launch");
    h->halo_set[0] = h->halo_set[1] = false;
    h->cur ^= 1;
    h->step += 1;
    return PF_OK;
}

int pf_get_clock(pf_handle* h, int64_t* step, int64_t* shifts) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (!step || !shifts) return fail(h, PF_EINVAL, "null output");
    *step = h->step;
    *shifts = h->shifts;
    return PF_OK;
}

int pf_set_clock(pf_handle* h, int64_t step, int64_t shifts) {
    if (!h) return fail(nullptr, PF_EINVAL, "null handle");
    if (int rc = split_closed(h)) return rc;
    if (step < 0 || shifts < 0) return fail(h, PF_EINVAL, "negative clock");
    h->step = step;
    h->shifts = shifts;
    h->have_front = false;
    return PF_OK;
}

}  // extern "C"
