/*
 * pf.h -- C ABI of libpf: the explicit time step of the variational
 * phase-field model of rapid alloy solidification of Mukherjee, Warren and
 * Voorhees (arXiv 2303.09671) on uniform 1D/2D/3D grids, on one GB300 GPU.
 *
 * The model (all quantities in the scaled units length W, time W^2/D_l,
 * concentration c0, energy density R T_m c0 / V_m):
 *   fields: phase field phi (1 solid, 0 liquid) and the separately evolved
 *   phase concentrations c_s, c_l (Sec. "Model", Eq. model1 with g = p);
 *   phase-field rate: Eq. phasefield_nonvar with the driving force
 *   DeltaG = f_s - f_l - mu_l (c_s - c_l) - D (c_s - c_l)(mu_s - mu_l),
 *   D = [M_s (1-p)(1 - A(1-p)) + A b M_l p^2] / Mbar (re-derived from
 *   Eq. model18 with the sources S_s = S_l = -A (c_s - c_l) of Sec.
 *   "Asymptotic analysis"; the printed Eq. drivingforce_nonvar has a sign/b typo);
 *   fluxes: the brackets of Eqs. cs_nonvar and cl_nonvar;
 *   interpolation: p(phi) of Eq. interpolation2, h_n of Eq. interpolation1;
 *   free energies: dilute ideal solution (Eqs. dil_linear, dil2, dil5) with
 *   mobilities M_i = D_i c_i (supplement, non-dimensionalisation);
 *   frozen temperature (Eq. ds1) and the moving window (Sec. "Numerical
 *   technique"); explicit finite differences on a staggered grid, forward
 *   Euler (Sec. "Numerical technique").
 *
 * Memory and ownership: a pf_handle owns every device buffer it allocates
 * (two ping-pong copies of the state in the chosen precision, SoA, x
 * fastest: phi, the mixture concentration c = p(phi) c_s + (1 - p(phi)) c_l,
 * the difference d = c_s - c_l and, in FP32, the low word of a compensated
 * c; plus reduction scratch).  pf_set_fields / pf_get_fields convert between
 * the caller's (phi, c_s, c_l) and this state.  Pointers passed to any call are borrowed
 * for the duration of that call only.  All device work is ordered on the
 * CUDA stream given to pf_create (a cudaStream_t passed as void*, NULL = the
 * legacy default stream); calls that return host values synchronise that
 * stream only.
 *
 * Errors: every int-returning call returns PF_OK (0) or a negative PF_E*
 * code; pf_last_error() gives a message owned by the handle.  No exception
 * and no abort crosses this boundary.
 */
#ifndef PF_H
#define PF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PF_OK = 0,
    PF_EINVAL = -1,        /* invalid argument or parameter */
    PF_ENOMEM = -2,        /* device or host allocation failed */
    PF_ECUDA = -3,         /* a CUDA runtime call failed */
    PF_ENONFINITE = -4,    /* a non-finite value was found in the fields */
    PF_ETIMEOUT = -5,      /* a bounded device wait ran out */
    PF_EUNSUPPORTED = -6   /* combination not supported by this build */
};
enum { PF_BC_NOFLUX = 0, PF_BC_PERIODIC = 1, PF_BC_DIRICHLET = 2, PF_BC_HALO = 3 };
enum { PF_FP32 = 0, PF_FP64 = 1 };
enum { PF_HOST = 0, PF_DEVICE = 1,
       /* pf_set_fields_step only: page-locked host memory read without a wait */
       PF_HOST_ASYNC = 2 };
enum { PF_INTERP_QUINTIC = 0, PF_INTERP_CUBIC = 1 };  /* h(phi), Sec. "Choice of interpolation functions" */
enum { PF_MOBILITY_DC = 0, PF_MOBILITY_CONST = 1 };   /* M_i = D_i c_i  or  M_i = D_i */

/* Uniform grid: dim in {1,2,3}; n[a] cells along axis a (x = axis 0 is the
 * fastest-varying index and the growth direction); unused axes must be 1;
 * dx the spacing in units of W. */
typedef struct {
    int dim;
    int64_t n[3];
    double dx;
} pf_grid;

/* Boundary conditions per axis side (Sec. "Numerical technique"):
 * PF_BC_NOFLUX   mirror ghosts and zero flux through the boundary face,
 * PF_BC_PERIODIC wrap (both sides of the axis must be periodic),
 * PF_BC_DIRICHLET fixed ghosts phi = dir_phi, c_s = dir_cs, c_l = dir_cl, whose
 *                phase-field rate is zero.  The same values fill the fresh
 *                layer of the moving window.
 * PF_BC_HALO     (3D, z sides only) the side borders another slab of a grid
 *                decomposed along z: the two ghost planes beyond it are held in
 *                the handle and imported with pf_set_halo before every step
 *                (see pf_get_halo). */
typedef struct {
    int lo[3], hi[3];
    double dir_phi, dir_cs, dir_cl;
} pf_bc;

/* Model and scheme parameters (scaled units).
 *   precision      PF_FP32 or PF_FP64 field storage and arithmetic (the
 *                  energy/solute reductions are always accumulated in FP64)
 *   interp         PF_INTERP_QUINTIC or PF_INTERP_CUBIC h(phi)
 *   lap_stencil    3 (1D), 5 or 9 (2D), 7 or 19 (3D) point Laplacian
 *   mobility_mode  PF_MOBILITY_DC or PF_MOBILITY_CONST
 *   H, sigma       well height and gradient coefficient (Eq. model1.1)
 *   M_phi          phase-field mobility (Eq. model12)
 *   D_s, D_l       phase diffusivities
 *   k_e            equilibrium partition coefficient, 0 < k_e < 1 (Eq. dil2)
 *   A              source/trapping parameter, S_s = S_l = -A (c_s - c_l)
 *   b, a           interpolation parameters of Eqs. interpolation1/2 (b > 0)
 *   delta          regularisation of 1/|grad phi|^2 -> 1/(|grad phi|^2 + delta^2)
 *   theta_ref, G_theta, v_pull, x0
 *                  frozen temperature in liquidus-concentration units,
 *                  theta(x,t) = theta_ref - G_theta ((x - x0) - v_pull t)   (Eq. ds1)
 *   dt             time step (must not exceed pf_stable_dt)
 *   c_inf          alloy composition (fresh window layer and k_v = c_inf/c_max)
 *   shift          1 = moving window along x (1D only): whenever v_pull t
 *                  reaches the next multiple of dx, drop the cold-end cell
 *                  and append a Dirichlet-valued cell at the hot end */
typedef struct {
    int precision;
    int interp;
    int lap_stencil;
    int mobility_mode;
    double H, sigma, M_phi, D_s, D_l, k_e, A, b, a, delta;
    double theta_ref, G_theta, v_pull, x0, dt, c_inf;
    int shift;
} pf_params;

typedef struct pf_handle pf_handle;

/* Validate the problem, allocate the device state on `stream` and set the
 * clock to step 0.  Fields are uninitialised until pf_set_fields.  Returns
 * PF_EINVAL for: dim outside 1..3, n[a] < 3 on an active axis or != 1 on an
 * inactive one, one-sided periodicity, dx <= 0, k_e outside (0,1), b <= 0,
 * H, sigma, M_phi, D_s, D_l <= 0, a stencil that does not match dim,
 * shift with dim != 1, dt <= 0 or dt above pf_stable_dt.
 *
 * The device state is (phi, c = p c_s + (1-p) c_l, d = c_s - c_l) in two
 * ping-pong copies; an FP32 state also keeps the low FP32 word of c, and in
 * 1D that of phi, so that both accumulate without rounding drift.  Two
 * environment variables, read here, select kernels for testing and tuning:
 * PF_GENERIC=1 runs 2D and 3D through the one-cell-per-thread kernel instead
 * of the paired two-lane kernels (a cross-check; same results to rounding),
 * PF_ZCHUNK=<planes> fixes the z-chunk of the 3D kernel,
 * PF_OVCHUNK=<planes> the slab length of pf_set_fields_step (default 16, at most
 * the z-chunk when that is fixed), PF_TMA=0 stages every plane of the 3D FP32
 * step with per-cell copies instead of tensor-memory-accelerator boxes (a
 * cross-check; identical results bit for bit; the boxes are used where n[0]
 * is a multiple of 4 and no x or y side is periodic), and
 * PF_TEST_DROP_COPIES=1 leaves the box copies out, so that the step's
 * bounded wait runs out (tests of PF_ETIMEOUT only). */
int pf_create(const pf_grid* grid, const pf_bc* bc, const pf_params* params,
              void* stream, pf_handle** out);

/* Copy the three fields in (pf_set_fields) or out (pf_get_fields).  Each
 * pointer addresses n[0]*n[1]*n[2] values of the handle's precision (float or
 * double), x fastest; where = PF_HOST (any host memory) or PF_DEVICE.  With
 * PF_HOST, pf_set_fields reads page-locked (pinned or registered) host memory
 * directly from the conversion kernel and stages other host memory through a
 * device copy; both synchronise the stream before returning, so the caller may
 * reuse its buffers at once.  pf_get_fields converts the state on the device
 * (into the idle state buffer for host outputs, which the copy engine then
 * reads out: a device-to-host copy runs at about twice the rate of a kernel
 * writing page-locked memory) and synchronises the stream. */
int pf_set_fields(pf_handle* h, const void* phi, const void* cs, const void* cl, int where);
int pf_get_fields(pf_handle* h, void* phi, void* cs, void* cl, int where);

/* pf_get_fields without the wait, for a pipeline that reads every step's
 * fields back while the next state is being uploaded.  The conversion of the
 * current state to (phi, c_s, c_l) is queued on an internal read-back stream
 * after the work already queued on the handle's stream: into device memory
 * (where = PF_DEVICE) directly, or into page-locked host memory (PF_HOST;
 * pageable memory returns PF_EINVAL) through a device staging buffer of the
 * handle's and the copy engine (two staging sets of 3 n[0]*n[1]*n[2] values,
 * used in turn so that a read-back's conversion need not wait for the
 * previous one's host copies, each allocated on first use; PF_ENOMEM if that
 * fails);
 * n[0]*n[1]*n[2] values each of the handle's precision.  The values are valid after pf_sync.
 * The handle keeps the state being read intact until the read-back has read
 * it: every later call that writes the state first orders itself after that
 * read (not after the copies to the host), except the upload of
 * pf_set_fields_step, which converts into the other state buffer and so
 * overlaps the read-back (only its step waits for the read).  The handle creates the
 * stream and its events on first use and frees them in pf_destroy. */
int pf_get_fields_async(pf_handle* h, void* phi, void* cs, void* cl, int where);

/* Wait for every piece of work of the handle, read-backs included.
 *
 * The 3D FP32 step waits on an mbarrier for the boxes of each plane, with a
 * time limit of half a second per wait.  A wait that runs out sets a device
 * flag of the handle, and the kernel finishes without waiting again (its
 * output state is then not valid).  pf_sync, pf_get_fields, pf_energy,
 * pf_solute_total, pf_front and pf_step_energies read the flag with the
 * synchronisation they already do: PF_ETIMEOUT once, after which the flag is
 * cleared. */
int pf_sync(pf_handle* h);

/* Advance n >= 0 forward-Euler steps (stream-ordered, no host sync). */
int pf_step(pf_handle* h, int64_t n);

/* pf_set_fields(h, phi, cs, cl, where) followed by pf_step(h, n), with the same
 * results bit for bit, for a state that arrives from the host before a run
 * (the forward-Euler step of Sec. "Numerical technique" applied to fields
 * read from page-locked host memory).  On a 3D grid of the paired kernel with
 * device memory or page-locked host memory and n >= 1, the fields are
 * converted slab by slab (16 planes each by default; the first step runs with
 * z-chunks of the same length, results being independent of it) on an internal
 * stream, and the first step of each chunk starts, on further internal
 * streams, as soon as the planes it reads (two below, one above the chunk,
 * wrapped on a periodic z axis) are in, so that stepping overlaps the
 * transfer.  From page-locked host memory the slabs are first copied by the
 * copy engine into a device staging buffer; those copies wait only for the
 * previous call's conversion of the same slab, not for its steps, so that
 * back-to-back calls keep the host link busy.  The handle's stream waits for
 * all of it; the remaining n - 1 steps follow on it.  where = PF_HOST_ASYNC:
 * page-locked host memory (PF_EINVAL otherwise) that the call does not wait
 * for; the caller keeps the buffers unchanged until pf_sync, or any other
 * call that synchronises the handle's stream, returns, so that a pipeline of
 * uploads and read-backs is queued without host round trips.  PF_HOST: returns
 * once the host buffers have been read (the
 * caller may reuse them); the steps may still be running.  Other grids,
 * pageable host memory or n = 0: the two calls in sequence.  The handle
 * creates its internal streams and events on first use and frees them in
 * pf_destroy.  Errors as pf_set_fields and pf_step; after PF_ECUDA the state
 * is undefined until the next pf_set_fields. */
int pf_set_fields_step(pf_handle* h, const void* phi, const void* cs, const void* cl, int where,
                       int64_t n);

/* ------------------------------------------------------------------------
 * Domain decomposition along z (3D): a grid split into slabs of whole x-y
 * planes, one handle per slab, each slab's z sides that border another slab
 * set to PF_BC_HALO.  The step's stencil reaches two planes across a face
 * (the face fluxes of Eqs. cs_nonvar / cl_nonvar need the phase-field rate of
 * the cells on both sides, which needs their neighbours), so before every
 * step each halo side imports the two planes beyond it from the neighbouring
 * slab: my low ghosts are the lower slab's two highest planes, my high ghosts
 * the upper slab's two lowest.  With the halos imported, a slab computes its
 * cells bit for bit as the undecomposed grid does, and the sums of the slabs'
 * pf_energy and pf_solute_total are the grid's (each gradient pair across a
 * slab boundary counted half in each slab).
 *
 * pf_halo_bytes: bytes of one side's halo (two planes of every state word:
 *   phi, c, d and, in FP32, the low word of c; 2 n[0] n[1] values each).
 * pf_get_halo: copy the two outermost planes of the current state at `side`
 *   (0 = low z, planes 0 and 1; 1 = high z, planes n[2]-2 and n[2]-1) into
 *   buf: field by field in the order above, each field's two planes in
 *   increasing z, x fastest, the handle's element type.
 * pf_set_halo: import the two ghost planes beyond `side` (low: planes -2, -1;
 *   high: n[2], n[2]+1) from buf, laid out as pf_get_halo writes them.
 * where = PF_DEVICE (device memory, stream-ordered) or PF_HOST (any host
 * memory; the call synchronises the stream).  `side` must be a PF_BC_HALO
 * side of the handle, else PF_EINVAL.
 *
 * On a handle with a halo side: pf_step advances one step at a time (n <= 1)
 * and needs every halo side imported since the last pf_set_fields or step;
 * pf_energy needs the same (its gradient pairs reach the ghost planes);
 * pf_solute_total, pf_front, pf_get_fields and pf_set_fields read the slab's
 * own cells only; pf_set_fields_step and pf_step_energies return PF_EINVAL.
 *
 * Split step, so that the halo exchange overlaps the step (3D, the fused 3D
 * kernel): pf_step_begin + pf_step_end advance one step exactly as
 * pf_step(h, 1) does, bit for bit (the forward-Euler step of Sec. "Numerical
 * technique").
 * - pf_step_begin queues the step's interior on a stream of the handle's own,
 *   ordered after the work already queued on the handle's stream.  The
 *   interior is the z-chunks of the fused kernel that read only planes
 *   0 .. n[2]-1 (chunks starting at plane >= 2 and ending at <= n[2]-2).
 *   It needs no halo.
 * - The caller then exports its boundary planes and imports its ghost planes
 *   (pf_get_halo, pf_set_halo; they read and write planes that the interior
 *   does not touch).
 * - pf_step_end queues the remaining chunks on the handle's stream, orders
 *   that stream after the interior, and advances the clock.  It needs every
 *   halo side imported, as pf_step does; if one is missing it returns
 *   PF_EINVAL and the split stays open, so the caller can import and call
 *   pf_step_end again.
 * Between the two calls pf_step, pf_step_begin, pf_set_fields,
 * pf_set_fields_step, pf_step_energies and pf_set_clock return PF_EINVAL.
 * Calls that only read the current state are allowed: the halos, the
 * fields, the diagnostics.  pf_step_end without an open split returns
 * PF_EINVAL, and so does pf_step_begin on a 1D or 2D grid or with the
 * generic kernel (PF_GENERIC).  The handle creates its interior stream on
 * first use and frees it in pf_destroy, which first waits for it.
 * ------------------------------------------------------------------------ */
int pf_halo_bytes(pf_handle* h, int64_t* bytes);
int pf_get_halo(pf_handle* h, int side, void* buf, int where);
int pf_set_halo(pf_handle* h, int side, const void* buf, int where);
int pf_step_begin(pf_handle* h);
int pf_step_end(pf_handle* h);

/* Discrete free energy of Eq. model1.1 for the current state, FP64:
 *   F_h = dV sum_i [H f_dw(phi_i) + p_i f_s,i + (1-p_i) f_l,i]
 *         + (sigma/2)(dV/dx^2) (1/2) sum_i sum_{j in stencil(i)} w_ij (phi_i - phi_j)^2,
 * w_ij the Laplacian weights, ghosts from the boundary conditions.
 * Synchronises the stream. */
int pf_energy(pf_handle* h, double* F);

/* Advance n >= 0 steps and record F_h (as pf_energy) after every step into
 * F[0..n-1] (caller-owned host memory).  The energies are reduced on the device
 * after each step and copied back once at the end, so the host does not wait
 * on every step (the planar-front run of Sec. "Numerical technique", which
 * checks the energy decrease of Eq. model1.1 step by step).  Without a moving
 * temperature or window the steps are replayed as captured 64-step CUDA
 * graphs on an internal stream ordered after and before the handle's.
 * Synchronises the stream once; PF_ENONFINITE if any record is not finite
 * (the steps are taken). */
int pf_step_energies(pf_handle* h, int64_t n, double* F);

/* Total solute S_h = dV sum_i [p_i c_s,i + (1-p_i) c_l,i] (Eq. model1), FP64.
 * Synchronises the stream. */
int pf_solute_total(pf_handle* h, double* S);

/* pf_solute_total without the wait: the reduction and the copy of S_h into *S
 * (page-locked host memory for the copy to be asynchronous; the caller owns it)
 * are queued on the handle's stream, and *S is valid once that stream has been
 * synchronised.  For a pipeline that reads every step's result without
 * stalling the next step's upload.  No finiteness check (the caller sees the
 * value); PF_EINVAL for a null handle or output, PF_ECUDA on a launch error. */
int pf_solute_total_async(pf_handle* h, double* S);

/* Front diagnostics: x_front = largest phi = 0.5 crossing along x over all
 * rows (linear interpolation, lab frame including window shifts; NaN when no
 * row has a crossing); v_front = (x_front - previous x_front)/(t - previous t)
 * from this handle's previous pf_front call (NaN on the first call or when no
 * time has passed); c_max = max of c = p c_s + (1-p) c_l, so that
 * k_v = c_inf / c_max (Sec. "Effect of parameter A on velocity-dependent
 * partition coefficient").  Synchronises the stream. */
int pf_front(pf_handle* h, double* x_front, double* v_front, double* c_max);

/* Clock of the handle (steps taken, window shifts); with pf_get_fields and
 * pf_set_fields this is a complete checkpoint. */
int pf_get_clock(pf_handle* h, int64_t* step, int64_t* shifts);
int pf_set_clock(pf_handle* h, int64_t step, int64_t shifts);

/* Explicit-Euler step bound used by pf_create's check (the paper states
 * none): min(dt_phi, dt_c) with lam = 4 dim / dx^2,
 * dt_phi = 2 / (M_phi (lam sigma + 2 H)), dt_c = 2 / (lam D_max), D_max the
 * largest concentration diffusivity q_n (p/c_s + (1-p)/c_l), M_s/c_s, M_l/c_l
 * over p in [0,1] at c_s = k_e c_inf, c_l = c_inf. */
int pf_stable_dt(const pf_grid* grid, const pf_params* params, double* dt);

/* ------------------------------------------------------------------------
 * Batched 1D pulled fronts: the k(V) sweep of Sec. "Effect of parameter A on
 * velocity-dependent partition coefficient" (k_v = c_inf / c_max at steady
 * state) for many instances of different lengths and pulling velocities in one
 * persistent launch per chunk of steps, replayed as a CUDA graph.
 *
 * Every instance is a 1D directional-solidification problem: frozen
 * temperature theta(x,t) = theta_ref - G_theta ((x - x0) - v t) (Eq. ds1, with
 * theta_ref, G_theta and x0 of `params` shared by all instances), no-flux
 * cold end, fixed hot end (bc.dir_*), moving window (Sec. "Numerical
 * technique"), and the shared model parameters of `params` (params.v_pull,
 * params.dt and params.shift are ignored; precision FP32 or FP64).
 * ------------------------------------------------------------------------ */
typedef struct {
    int n_instances;
    const int64_t* n;      /* cells per instance, 8..8192 (FP32) or 8..4096 (FP64) */
    const double* v_pull;  /* pulling velocity per instance, >= 0 */
    const double* dt;      /* time step per instance; NULL or <= 0: 0.9 pf_stable_dt
                              capped at 0.5 dx / v */
    const void* phi0;      /* initial fields, instances packed one after another,  */
    const void* cs0;       /* host memory, element type of params.precision        */
    const void* cl0;
    double dx;
    pf_bc bc;              /* lo[0] must be PF_BC_NOFLUX; hi[0] PF_BC_DIRICHLET, or
                              PF_BC_NOFLUX for closed boxes without a moving window
                              (all v_pull = 0), e.g. the planar front of Sec.
                              "Numerical technique" with F_h recorded every step */
    pf_params params;
    int64_t max_steps;         /* per instance */
    int64_t steps_per_launch;  /* steps of one persistent launch (> 0) */
    int launches_per_graph;    /* launches captured in one CUDA graph (> 0) */
    int64_t check_every;       /* steps between k_v evaluations (> 0) */
    double window;             /* minimum time between the two k_v samples of a rate */
    double tol;                /* converged when |dk_v/dt| < tol ...                  */
    double min_travel;         /* ... and the temperature has been pulled >= min_travel
                                  (units of W), i.e. t >= min_travel / v */
    int cells_per_thread;      /* 1, 2, 4 or 8; 0 = autotune */
    int64_t energy_every;      /* > 0: record the free energy F_h (as pf_energy
                                  computes it) after every energy_every-th step,
                                  in FP64 inside the persistent launch; 0: none */
} pf_batch_desc;

typedef struct {
    double* k_v;           /* per instance: last k_v = c_inf / c_max; NaN where the
                              state stopped being finite (that instance then stops,
                              with converged = 0) */
    double* dkdt;          /* per instance: last |dk_v/dt| */
    double* t;             /* per instance: simulated time reached */
    int64_t* steps;        /* per instance: steps taken */
    int* converged;        /* per instance: 1 if converged */
    void* phi;             /* optional (may be NULL): packed final fields, host */
    void* cs;
    void* cl;
    int cells_per_thread;  /* the value used (autotuned or given) */
    int64_t launches;      /* batch-kernel launches issued */
    double gpu_ms;         /* device time of the stepping (CUDA events) */
    double* energy;        /* optional (may be NULL), with energy_every > 0: host
                              array [n_instances][max_steps / energy_every] of F_h
                              records; NaN where an instance had stopped */
} pf_batch_result;

/* Run the batch until every instance has converged or taken max_steps
 * steps.  All arrays are caller-owned host memory of n_instances entries (the
 * optional field arrays hold the sum of n).  Allocates and frees its own device
 * memory; synchronises `stream`.  Returns PF_EINVAL for invalid descriptors. */
int pf_run_batch(const pf_batch_desc* desc, pf_batch_result* res, void* stream);

/* ------------------------------------------------------------------------
 * Parameter sensitivities of the pulled-front partition coefficient, for
 * calibrating the trapping parameter A, the mobility shape b and the
 * phase-field mobility M_phi against a k(V) target (the tuning of A, b and W
 * of Sec. "Tailoring the partition coefficient: Selection of A").
 *
 * For every instance of `batch` (same meaning as for pf_run_batch; the
 * k_v-convergence fields are ignored) the run takes exactly `nsteps` steps
 * and evaluates k_i = c_inf / max_x c, c = p c_s + (1-p) c_l, at the end.
 * The derivatives dk_i/dtheta are exact derivatives of the discrete run; at
 * the maximum the derivative of the maximising cell is taken (a subgradient
 * where two cells tie).  Two ways to the same numbers:
 *   PF_ADJ_TANGENT  tangent-linear: the state is carried as value + derivative
 *                   along one parameter, one CTA per instance and parameter,
 *                   all concurrent;
 *   PF_ADJ_REVERSE  reverse sweep: the forward run stores its state every
 *                   checkpoint_every steps (0: ceil(sqrt(nsteps)), at most 1024);
 *                   each segment is then re-run recording every step and swept
 *                   backwards with the adjoint of the fused step, from
 *                   d k_i / d c at the maximum, one CTA per instance.  The cost
 *                   does not grow with the number of parameters.
 * With k_target given, the loss is
 *   L = sum_i (k_i - k_target_i)^2,  dL/dtheta = sum_i 2 (k_i - k_target_i) dk_i/dtheta.
 * batch.params.precision selects FP32 or FP64 arithmetic for value and
 * derivative; instances hold at most 4096 (FP32) or 2048 (FP64) cells.
 * ------------------------------------------------------------------------ */
enum { PF_ADJ_MPHI = 1, PF_ADJ_A = 2, PF_ADJ_B = 4 };
enum { PF_ADJ_TANGENT = 0, PF_ADJ_REVERSE = 1 };

typedef struct {
    pf_batch_desc batch;      /* instances, initial fields, shared parameters */
    int64_t nsteps;           /* steps per instance (> 0) */
    int wrt;                  /* parameters to differentiate: PF_ADJ_* bits (non-zero) */
    const double* k_target;   /* per instance, host; NULL: loss and grad are 0 */
    int mode;                 /* PF_ADJ_TANGENT or PF_ADJ_REVERSE */
    int checkpoint_every;     /* PF_ADJ_REVERSE: steps between stored states (0: automatic) */
} pf_adjoint_desc;

typedef struct {
    double* k;                /* optional [n_instances]: k_i after nsteps */
    double* dk;               /* optional [3 * n_instances]: dk_i/d(M_phi, A, b) at
                                 dk[3 i + j]; 0 for parameters not in wrt */
    double loss;              /* L (0 without k_target) */
    double grad[3];           /* dL/d(M_phi, A, b) (0 outside wrt or without k_target) */
    double gpu_ms;            /* device time of the stepping (CUDA events) */
} pf_adjoint_result;

/* Run the instances with derivatives and fill `res`.  Caller-owned host
 * arrays; allocates and frees its own device memory; synchronises `stream`.
 * PF_EINVAL for invalid descriptors (empty wrt, nsteps <= 0, instance too long,
 * the conditions of pf_run_batch). */
int pf_adjoint(const pf_adjoint_desc* desc, pf_adjoint_result* res, void* stream);

/* Allocation-free FP64 free energy and total solute (the paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory -- a process whose device memory is held by another allocator, a
 * monitoring or real-time path that must not block or fail on cudaMalloc, or a
 * caller without a pf_handle, since pf_create allocates).
 *
 * Computes F_h (out[0]) and S_h (out[1]) as pf_energy and pf_solute_total do
 * (the same reduction kernel and grid), directly from caller-owned device
 * arrays phi, cs, cl of n[0]*n[1]*n[2] values (x fastest, element type of
 * params->precision: float for PF_FP32, double for PF_FP64) at the clock
 * (step, shifts), and writes the two doubles to the caller-owned device
 * pointer `out` (at least 2 doubles), ordered on `stream` (no host
 * synchronisation).  It calls no cudaMalloc/cudaFree: the reduction's block
 * partials live in a 32 KiB file-scope device array that stays resident on
 * every GPU that loads the library.  Every call looks the array's device
 * address up (cudaGetSymbolAddress, no allocation); the first call on a
 * device also loads the library's device code there, so make it before any
 * stream capture on that device.  All calls share the array; each call
 * rewrites every partial it reads, but calls whose kernels overlap on the GPU
 * race and must be serialised by the caller.  Returns PF_EINVAL (message via
 * pf_last_error(NULL)) for null pointers, a negative clock, grids above 2^30
 * cells, and every description pf_create rejects except for the conditions
 * that concern stepping only (dt above the stability bound, the moving
 * window, the 2D/3D step-launch limits); dt must be finite.  The pointers
 * themselves cannot be checked here: they must address device memory of the
 * sizes above. */
int pf_energy_solute_noalloc(const pf_grid* grid, const pf_bc* bc, const pf_params* params,
                             int64_t step, int64_t shifts, const void* phi, const void* cs,
                             const void* cl, double* out, void* stream);

/* Message describing the last error on h (or the last pf_create failure when
 * h is NULL).  Owned by the library; valid until the next call on h. */
const char* pf_last_error(pf_handle* h);

/* Free the handle and its device memory (stream-ordered). */
void pf_destroy(pf_handle* h);

#ifdef __cplusplus
}
#endif
#endif
