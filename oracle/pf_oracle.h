/*
 * pf_oracle.h -- plain FP64 CPU oracle for the explicit time step of the
 * variational phase-field model of rapid alloy solidification
 * (Mukherjee, Warren & Voorhees, arXiv 2303.09671).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no source with the CUDA library.
 *
 * What it computes (all in the scaled units: length W, time W^2/D_l,
 * concentration c0, energy density R T_m c0 / V_m):
 *   - the phase-field rate of Eq. phasefield_nonvar with the driving force
 *     re-derived from Eq. model18 (the printed Eq. drivingforce_nonvar carries
 *     a sign/b typo; a test plants the printed form and shows it breaks the
 *     energy law of Eqs. model10-model12),
 *   - the solid and liquid fluxes, i.e. the brackets of Eqs. cs_nonvar and
 *     cl_nonvar, on a staggered grid (Sec. "Numerical technique"),
 *   - forward-Euler updates of (c, d) = (p c_s + (1-p) c_l, c_s - c_l), which
 *     are Eqs. model5/model6 and the difference of Eqs. cs_nonvar/cl_nonvar,
 *     or (form = 1) the literal c_s, c_l updates with their source terms,
 *   - the dilute ideal-solution free energies of Eqs. dil_linear/dil2/dil5,
 *   - the frozen temperature of Eq. ds1 and the moving window of the
 *     "Numerical technique" section (1D only),
 *   - FP64 diagnostics: discrete free energy (Eq. model1.1), total solute,
 *     the phi = 0.5 front and c_max (k_v = c_inf / c_max).
 *
 * Parity pins for every function are listed in the test files
 * tests/test_oracle_*.py; "parity unpinned" is stated there where none exists.
 */
#ifndef PF_ORACLE_H
#define PF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_NOFLUX = 0, ORC_BC_PERIODIC = 1, ORC_BC_DIRICHLET = 2 };

typedef struct {
    int dim;              /* 1, 2 or 3 */
    int64_t n[3];         /* cells per axis; x fastest; unused axes = 1 */
    double dx;            /* uniform spacing (units of W) */
    int bc_lo[3], bc_hi[3];
    double dir_phi, dir_cs, dir_cl;   /* Dirichlet ghost values / fresh layer */
    int interp;           /* 0: quintic h, 1: cubic h */
    int lap;              /* 3 (1D), 5 or 9 (2D), 7 or 19 (3D) */
    int mobility;         /* 0: M_i = D_i c_i ; 1: M_i = D_i (constant) */
    double H, sigma, M_phi, D_s, D_l, k_e, A, b, a, delta;
    double theta_ref, G_theta, v_pull, x0;   /* theta(x,t) of Eq. ds1 */
    double dt, c_inf;
    int shift;            /* 1D moving window on/off */
    int form;             /* 0: conservative (c,d) update; 1: literal c_s,c_l */
    int plant;            /* TEST ONLY: bitmask of deliberately planted mistakes */
} orc_params;

typedef struct {
    int64_t step;         /* steps taken; t = step * dt */
    int64_t shifts;       /* window shifts taken (1D pulled front) */
} orc_clock;

/* Pointwise quantities at one cell.  out[] receives, in order:
 * 0 p, 1 p', 2 f_dw, 3 f_dw', 4 mu_s, 5 mu_l, 6 f_s, 7 f_l, 8 M_s, 9 M_l,
 * 10 Mbar, 11 drag D, 12 DeltaG, 13 q_n, 14 w_s, 15 w_l, 16 h_n, 17 a(phi),
 * 18 Y.   Returns 0. */
int orc_point(const orc_params* P, double phi, double cs, double cl,
              double theta, double* out);

/* Rates of the state (phi, cs, cl) at the time of clk: phidot, cdot = div F_c,
 * ddot = div F_d on every cell (any pointer may be NULL). */
int orc_rates(const orc_params* P, const orc_clock* clk, const double* phi,
              const double* cs, const double* cl, double* phidot,
              double* cdot, double* ddot);

/* Advance nsteps forward-Euler steps in place.  If energy is non-NULL it
 * receives the discrete free energy of the state BEFORE each step
 * (nsteps values).  Returns 0, or -1 on invalid arguments, -2 on a
 * non-finite value. */
int orc_step(const orc_params* P, orc_clock* clk, double* phi, double* cs,
             double* cl, int64_t nsteps, double* energy);

double orc_energy(const orc_params* P, const orc_clock* clk, const double* phi,
                  const double* cs, const double* cl);
double orc_solute(const orc_params* P, const double* phi, const double* cs,
                  const double* cl);
/* p(phi) and the mixture c = p c_s + (1 - p) c_l of each of n cells (either
 * output may be NULL).  Returns 0, or -1 on invalid arguments. */
int orc_mixture(const orc_params* P, const double* phi, const double* cs,
                const double* cl, int64_t n, double* p_out, double* c_out);
/* front position (lab frame, largest phi=0.5 crossing along x over all rows)
 * and c_max.  x_front = NaN when no row has a crossing. */
int orc_front(const orc_params* P, const orc_clock* clk, const double* phi,
              const double* cs, const double* cl, double* x_front,
              double* c_max);

int orc_num_threads(void);
int orc_set_threads(int n);   /* threads of later sweeps (n <= 0: unchanged); returns the count */

#ifdef __cplusplus
}
#endif
#endif
