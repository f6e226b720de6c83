/*
 * pf_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see
 * pf_oracle.h).  Written for clarity, not speed: every step of the discrete
 * method is a separate loop over a ghost-padded array, in the order
 *   ghosts -> pointwise values -> phase-field rate -> face fluxes -> update,
 * with OpenMP only over the outermost loop of each sweep.
 *
 * The discrete method (Sec. "Numerical technique": explicit finite
 * differences on a staggered grid, second order in space, forward Euler):
 *   cells hold phi, c_s, c_l; faces hold the fluxes; face values of phi, c_s,
 *   c_l, d and phidot are the means of the two cells; the interpolation
 *   functions are evaluated at the face phi; the face gradient is the
 *   one-sided difference along the face normal and the mean of the two cells'
 *   centred differences across it; 1/|grad phi|^2 is regularised as
 *   1/(|grad phi|^2 + delta^2).
 */
#include "pf_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* planted mistakes (tests only) */
#define PLANT_PRINTED_DRAG   1   /* use the drag coefficient exactly as printed */
#define PLANT_NO_ANTITRAP    2   /* drop the (1-A) d phidot terms of the fluxes */
#define PLANT_NO_CROSS       4   /* drop the cross term of the phi equation */
#define PLANT_NO_K           8   /* drop the (1-A)^2 d^2 term of the phi-rate coefficient */
#define PLANT_TANG_SIGN     16   /* wrong sign of the tangential projection */
#define PLANT_SWAP_W        32   /* swap the solid/liquid anti-trapping weights */
#define PLANT_MU_S_CRYST    64   /* crystallisation force with mu_s instead of mu_l */
/* planted mistakes of the diagnostics and the moving window (tests only) */
#define PLANT_FRONT_INDEX  128   /* phi = 0.5 crossing placed one cell too low */
#define PLANT_FRONT_HALF   256   /* crossing measured from the cell edge, not its centre */
#define PLANT_FRESH_CINF   512   /* fresh hot-end layer with c_s = c_inf instead of the Dirichlet c_s */
#define PLANT_SHIFT_EARLY 1024   /* window shifted once v t exceeds shifts dx (one shift ahead) */

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following sweeps (n <= 0: leave unchanged); returns the
 * number in use afterwards. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---------------------------------------------------------------- pointwise */

/* h(phi): quintic or cubic (Sec. "Choice of interpolation functions") */
static double h_of(const orc_params* P, double f) {
    if (P->interp == 1) return f * f * (3.0 - 2.0 * f);
    return f * f * f * (6.0 * f * f - 15.0 * f + 10.0);
}
static double dh_of(const orc_params* P, double f) {
    if (P->interp == 1) return 6.0 * f * (1.0 - f);
    return 30.0 * f * f * (1.0 - f) * (1.0 - f);
}
/* p(phi) = h + a (phi - 1/2) phi^2 (1-phi)^2   (Eq. interpolation2) */
static double p_of(const orc_params* P, double f) {
    return h_of(P, f) + P->a * (f - 0.5) * f * f * (1.0 - f) * (1.0 - f);
}
static double dp_of(const orc_params* P, double f) {
    double w = f * f * (1.0 - f) * (1.0 - f);
    double dw = 2.0 * f * (1.0 - f) * (1.0 - 2.0 * f);
    return dh_of(P, f) + P->a * (w + (f - 0.5) * dw);
}
/* double well f_dw = phi^2 (1-phi)^2 (Eq. model1.1) and its derivative */
static double fdw_of(double f) { return f * f * (1.0 - f) * (1.0 - f); }
static double dfdw_of(double f) { return 2.0 * f * (1.0 - f) * (1.0 - 2.0 * f); }

/* diffusion potentials of the dilute ideal solution (Eqs. dil_linear, dil2):
 * with eps_l = 0, eps_s = ln(1/k_e), mu_s = ln(c_s / k_e), mu_l = ln c_l */
static double mu_s_of(const orc_params* P, double cs) { return log(cs) - log(P->k_e); }
static double mu_l_of(double cl) { return log(cl); }
/* bulk free energies (Eq. dil_linear; f_s^A - f_l^A from Eq. dil5 with
 * c_l^eq = theta, f_l^A = 0; the common linear term c ln c0 is dropped) */
static double fs_of(const orc_params* P, double cs, double theta) {
    return -(1.0 - P->k_e) * theta + cs * log(1.0 / P->k_e) + cs * log(cs) - cs;
}
static double fl_of(double cl) { return cl * log(cl) - cl; }

/* mobilities M_i = D_i dc_i/dmu_i = D_i c_i (supplement, non-dimensionalisation) */
static double Ms_of(const orc_params* P, double cs) {
    return P->mobility == 1 ? P->D_s : P->D_s * cs;
}
static double Ml_of(const orc_params* P, double cl) {
    return P->mobility == 1 ? P->D_l : P->D_l * cl;
}

/* drag coefficient D(phi): from Eq. model18 with S_s = S_l = -A(c_s-c_l),
 * g = p, M_s^n = M_s/h_n, M_l^n = M_l/(1-h_n) (Eqs. normal2, interpolation1):
 *   D = [M_s (1-p)(1 - A(1-p)) + A b M_l p^2] / Mbar,
 * Mbar = M_s (1-p) + b M_l p (text after Eq. drivingforce_nonvar). */
static double drag_of(const orc_params* P, double p, double Ms, double Ml) {
    double Mbar = Ms * (1.0 - p) + P->b * Ml * p;
    if (P->plant & PLANT_PRINTED_DRAG)   /* Eq. drag_coefficient as printed */
        return (Ms * (1.0 - p) * (P->A * (1.0 - p) - 1.0) - Ml * p * P->A * p) /
               (Ms * (1.0 - p) + Ml * p);
    return (Ms * (1.0 - p) * (1.0 - P->A * (1.0 - p)) + P->A * P->b * Ml * p * p) / Mbar;
}

/* driving force DeltaG = f_s - f_l - mu_l (c_s - c_l) - D (c_s - c_l)(mu_s - mu_l)
 * (Eqs. free_energy2-free_energy4 with the re-derived D) */
static double dG_of(const orc_params* P, double p, double cs, double cl, double theta) {
    double mus = mu_s_of(P, cs), mul = mu_l_of(cl);
    double d = cs - cl;
    double D = drag_of(P, p, Ms_of(P, cs), Ml_of(P, cl));
    double muc = (P->plant & PLANT_MU_S_CRYST) ? mus : mul;
    return fs_of(P, cs, theta) - fl_of(cl) - muc * d - D * d * (mus - mul);
}

int orc_point(const orc_params* P, double phi, double cs, double cl,
              double theta, double* out) {
    double p = p_of(P, phi);
    double Ms = Ms_of(P, cs), Ml = Ml_of(P, cl);
    double Mbar = Ms * (1.0 - p) + P->b * Ml * p;
    double hn = P->b * p / (P->b * p + 1.0 - p);
    out[0] = p;
    out[1] = dp_of(P, phi);
    out[2] = fdw_of(phi);
    out[3] = dfdw_of(phi);
    out[4] = mu_s_of(P, cs);
    out[5] = mu_l_of(cl);
    out[6] = fs_of(P, cs, theta);
    out[7] = fl_of(cl);
    out[8] = Ms;
    out[9] = Ml;
    out[10] = Mbar;
    out[11] = drag_of(P, p, Ms, Ml);
    out[12] = dG_of(P, p, cs, cl, theta);
    out[13] = Ms * Ml * (P->b * p + 1.0 - p) / Mbar;            /* q_n, Eq. normal2 */
    out[14] = Ms * (1.0 - p) / Mbar;                            /* M_s^n / (M_s^n+M_l^n) */
    out[15] = P->b * Ml * p / Mbar;                             /* M_l^n / (M_s^n+M_l^n) */
    out[16] = hn;                                               /* Eq. interpolation1 */
    out[17] = (Ms - P->b * Ml) * p * (1.0 - p) / Mbar;          /* Eq. shape_function */
    out[18] = p * out[4] + (1.0 - p) * out[5];
    return 0;
}

/* ---------------------------------------------------------------- grid */

typedef struct {
    int64_t n[3], g[3], P[3];   /* interior size, ghost width, padded size */
    int64_t s[3];               /* padded strides */
    int64_t total;
} layout;

static void make_layout(const orc_params* P, layout* L) {
    for (int a = 0; a < 3; ++a) {
        L->n[a] = (a < P->dim) ? P->n[a] : 1;
        L->g[a] = (a < P->dim) ? 2 : 0;
        L->P[a] = L->n[a] + 2 * L->g[a];
    }
    L->s[0] = 1;
    L->s[1] = L->P[0];
    L->s[2] = L->P[0] * L->P[1];
    L->total = L->P[0] * L->P[1] * L->P[2];
}
static int64_t pidx(const layout* L, int64_t i, int64_t j, int64_t k) {
    return ((k + L->g[2]) * L->P[1] + (j + L->g[1])) * L->P[0] + (i + L->g[0]);
}
static int64_t uidx(const layout* L, int64_t i, int64_t j, int64_t k) {
    return (k * L->n[1] + j) * L->n[0] + i;
}
/* map a possibly-ghost coordinate to the interior one; -1 = Dirichlet ghost */
static int64_t map_axis(const orc_params* P, const layout* L, int a, int64_t i) {
    int64_t n = L->n[a];
    if (i >= 0 && i < n) return i;
    int bc = (i < 0) ? P->bc_lo[a] : P->bc_hi[a];
    if (bc == ORC_BC_PERIODIC) return (i < 0) ? i + n : i - n;
    if (bc == ORC_BC_NOFLUX) return (i < 0) ? -i - 1 : 2 * n - 1 - i;
    return -1;
}

/* fill a padded copy of an unpadded field; Dirichlet ghosts take dval */
static void pad_field(const orc_params* P, const layout* L, const double* u,
                      double* pf, double dval) {
#pragma omp parallel for schedule(static)
    for (int64_t k = -L->g[2]; k < L->n[2] + L->g[2]; ++k)
        for (int64_t j = -L->g[1]; j < L->n[1] + L->g[1]; ++j)
            for (int64_t i = -L->g[0]; i < L->n[0] + L->g[0]; ++i) {
                int64_t mi = map_axis(P, L, 0, i), mj = map_axis(P, L, 1, j),
                        mk = map_axis(P, L, 2, k);
                pf[pidx(L, i, j, k)] = (mi < 0 || mj < 0 || mk < 0)
                                           ? dval : u[uidx(L, mi, mj, mk)];
            }
}

/* Laplacian stencil: offsets and weights in units of 1/dx^2, centre excluded.
 * 3: [1,-2,1]; 5/7: nearest neighbours; 9: faces 2/3, corners 1/6;
 * 19: faces 1/3, edges 1/6.  Returns the number of entries. */
static int lap_stencil(int lap, int off[18][3], double w[18]) {
    int m = 0;
    if (lap == 3 || lap == 5 || lap == 7) {
        int na = (lap == 3) ? 1 : (lap == 5 ? 2 : 3);
        for (int a = 0; a < na; ++a)
            for (int s = -1; s <= 1; s += 2) {
                off[m][0] = off[m][1] = off[m][2] = 0;
                off[m][a] = s; w[m] = 1.0; ++m;
            }
        return m;
    }
    if (lap == 9) {
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy) continue;
                off[m][0] = dx; off[m][1] = dy; off[m][2] = 0;
                w[m] = (dx && dy) ? 1.0 / 6.0 : 2.0 / 3.0; ++m;
            }
        return m;
    }
    /* 19 */
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int nz = (dx != 0) + (dy != 0) + (dz != 0);
                if (nz == 0 || nz == 3) continue;
                off[m][0] = dx; off[m][1] = dy; off[m][2] = dz;
                w[m] = (nz == 1) ? 1.0 / 3.0 : 1.0 / 6.0; ++m;
            }
    return m;
}

/* frozen temperature (Eq. ds1) in liquidus-concentration units:
 * theta = theta_ref - G_theta ((x - x0) - v_pull t), x the lab coordinate of the
 * cell centre along axis 0 */
static double theta_at(const orc_params* P, const orc_clock* clk, int64_t i) {
    double t = (double)clk->step * P->dt;
    double x = ((double)i + 0.5) * P->dx + (double)clk->shifts * P->dx;
    return P->theta_ref - P->G_theta * ((x - P->x0) - P->v_pull * t);
}

static int valid_params(const orc_params* P) {
    if (P->dim < 1 || P->dim > 3) return 0;
    for (int a = 0; a < P->dim; ++a) {
        if (P->n[a] < 3) return 0;
        if ((P->bc_lo[a] == ORC_BC_PERIODIC) != (P->bc_hi[a] == ORC_BC_PERIODIC)) return 0;
    }
    if (!(P->dx > 0) || !(P->k_e > 0 && P->k_e < 1) || !(P->b > 0)) return 0;
    if (P->dim == 1 && P->lap != 3) return 0;
    if (P->dim == 2 && P->lap != 5 && P->lap != 9) return 0;
    if (P->dim == 3 && P->lap != 7 && P->lap != 19) return 0;
    if (P->shift && P->dim != 1) return 0;
    return 1;
}

/* ---------------------------------------------------------------- work arrays */

typedef struct {
    layout L;
    double *phi, *cs, *cl;       /* padded raw fields */
    double *p, *mus, *mul, *Y;   /* padded pointwise values */
    double *pd;                  /* padded phase-field rate */
    double *Fa[3], *Fb[3];       /* face fluxes per axis: (F_c,F_d) or (F_s,F_l) */
    int64_t fn[3][3];            /* face-array sizes per axis */
} work;

static void work_free(work* W) {
    free(W->phi); free(W->cs); free(W->cl);
    free(W->p); free(W->mus); free(W->mul); free(W->Y); free(W->pd);
    for (int a = 0; a < 3; ++a) { free(W->Fa[a]); free(W->Fb[a]); }
}
static int work_alloc(const orc_params* P, work* W) {
    memset(W, 0, sizeof(*W));
    make_layout(P, &W->L);
    int64_t T = W->L.total;
    W->phi = malloc(T * sizeof(double)); W->cs = malloc(T * sizeof(double));
    W->cl = malloc(T * sizeof(double)); W->p = malloc(T * sizeof(double));
    W->mus = malloc(T * sizeof(double)); W->mul = malloc(T * sizeof(double));
    W->Y = malloc(T * sizeof(double)); W->pd = malloc(T * sizeof(double));
    int ok = W->phi && W->cs && W->cl && W->p && W->mus && W->mul && W->Y && W->pd;
    for (int a = 0; a < P->dim; ++a) {
        for (int b = 0; b < 3; ++b) W->fn[a][b] = W->L.n[b] + (a == b ? 1 : 0);
        int64_t F = W->fn[a][0] * W->fn[a][1] * W->fn[a][2];
        W->Fa[a] = malloc(F * sizeof(double));
        W->Fb[a] = malloc(F * sizeof(double));
        ok = ok && W->Fa[a] && W->Fb[a];
    }
    if (!ok) { work_free(W); return -1; }
    return 0;
}
static int64_t fidx(const work* W, int a, int64_t fi, int64_t j, int64_t k) {
    /* face index along axis a: cell coordinate of the face's left cell + 1 */
    return (k * W->fn[a][1] + j) * W->fn[a][0] + fi;
}

/* centred difference of padded field f at padded index c along axis a */
static double cgrad(const work* W, const double* f, int64_t c, int a, double dx) {
    return (f[c + W->L.s[a]] - f[c - W->L.s[a]]) / (2.0 * dx);
}

/* ghosts + pointwise values on the whole padded domain */
static void stage_fields(const orc_params* P, work* W, const double* phi,
                         const double* cs, const double* cl) {
    pad_field(P, &W->L, phi, W->phi, P->dir_phi);
    pad_field(P, &W->L, cs, W->cs, P->dir_cs);
    pad_field(P, &W->L, cl, W->cl, P->dir_cl);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < W->L.total; ++c) {
        W->p[c] = p_of(P, W->phi[c]);
        W->mus[c] = mu_s_of(P, W->cs[c]);
        W->mul[c] = mu_l_of(W->cl[c]);
        W->Y[c] = W->p[c] * W->mus[c] + (1.0 - W->p[c]) * W->mul[c];
    }
}

/* phase-field rate (Eq. phasefield_nonvar with the re-derived driving force):
 *   K phidot = sigma L_h phi - H f_dw' - DeltaG p'
 *              + (1-A) d p (1-p)/Mbar (M_s grad mu_s - b M_l grad mu_l).grad phi r
 *   K = 1/M_phi + (1-A)^2 d^2 b p (1-p) r / (Mbar (b p + 1 - p)),
 *   r = 1/(|grad phi|^2 + delta^2), gradients centred. */
static void stage_phidot(const orc_params* P, const orc_clock* clk, work* W) {
    const layout* L = &W->L;
    int off[18][3]; double wl[18];
    int m = lap_stencil(P->lap, off, wl);
    double dx = P->dx, A = P->A, b = P->b;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < L->n[2]; ++k)
        for (int64_t j = 0; j < L->n[1]; ++j)
            for (int64_t i = 0; i < L->n[0]; ++i) {
                int64_t c = pidx(L, i, j, k);
                double f = W->phi[c], cs = W->cs[c], cl = W->cl[c];
                double p = W->p[c], dp = dp_of(P, f);
                double Ms = Ms_of(P, cs), Ml = Ml_of(P, cl);
                double Mbar = Ms * (1.0 - p) + b * Ml * p;
                double d = cs - cl;
                double theta = theta_at(P, clk, i);
                double lap = 0.0;
                for (int e = 0; e < m; ++e) {
                    int64_t o = off[e][0] * L->s[0] + off[e][1] * L->s[1] + off[e][2] * L->s[2];
                    lap += wl[e] * (W->phi[c + o] - f);
                }
                lap /= dx * dx;
                double g2 = 0.0, cross = 0.0;
                for (int a = 0; a < P->dim; ++a) {
                    double gp = cgrad(W, W->phi, c, a, dx);
                    double gs = cgrad(W, W->mus, c, a, dx);
                    double gl = cgrad(W, W->mul, c, a, dx);
                    g2 += gp * gp;
                    cross += (Ms * gs - b * Ml * gl) * gp;
                }
                double r = 1.0 / (g2 + P->delta * P->delta);
                double K = 1.0 / P->M_phi;
                if (!(P->plant & PLANT_NO_K))
                    K += (1.0 - A) * (1.0 - A) * d * d * b * p * (1.0 - p) * r /
                         (Mbar * (b * p + 1.0 - p));
                double R = P->sigma * lap - P->H * dfdw_of(f) - dG_of(P, p, cs, cl, theta) * dp;
                if (!(P->plant & PLANT_NO_CROSS))
                    R += (1.0 - A) * d * p * (1.0 - p) / Mbar * cross * r;
                W->pd[c] = R / K;
            }
    /* ghost rates: copies for no-flux / periodic, zero for a fixed (Dirichlet) ghost */
#pragma omp parallel for schedule(static)
    for (int64_t k = -L->g[2]; k < L->n[2] + L->g[2]; ++k)
        for (int64_t j = -L->g[1]; j < L->n[1] + L->g[1]; ++j)
            for (int64_t i = -L->g[0]; i < L->n[0] + L->g[0]; ++i) {
                if (i >= 0 && i < L->n[0] && j >= 0 && j < L->n[1] && k >= 0 && k < L->n[2])
                    continue;
                int64_t mi = map_axis(P, L, 0, i), mj = map_axis(P, L, 1, j),
                        mk = map_axis(P, L, 2, k);
                W->pd[pidx(L, i, j, k)] = (mi < 0 || mj < 0 || mk < 0)
                                              ? 0.0 : W->pd[pidx(L, mi, mj, mk)];
            }
}

/* face fluxes between padded cells cL and cR = cL + e_a (brackets of
 * Eqs. cs_nonvar and cl_nonvar; F = -J):
 *   F_s = q g_a (g.grad Y) r + M_s [d_a mu_s - g_a (g.grad mu_s) r] + (1-A) d w_s phidot g_a r
 *   F_l = q g_a (g.grad Y) r + M_l [d_a mu_l - g_a (g.grad mu_l) r] - (1-A) d w_l phidot g_a r */
static void face_flux(const orc_params* P, const work* W, int64_t cL, int64_t cR,
                      int a, double* Fs, double* Fl, double* pf_out) {
    double dx = P->dx, A = P->A, b = P->b;
    double f = 0.5 * (W->phi[cL] + W->phi[cR]);
    double cs = 0.5 * (W->cs[cL] + W->cs[cR]);
    double cl = 0.5 * (W->cl[cL] + W->cl[cR]);
    double d = cs - cl;
    double pdot = 0.5 * (W->pd[cL] + W->pd[cR]);
    double p = p_of(P, f);
    double Ms = Ms_of(P, cs), Ml = Ml_of(P, cl);
    double Mbar = Ms * (1.0 - p) + b * Ml * p;
    double q = Ms * Ml * (b * p + 1.0 - p) / Mbar;
    double ws = Ms * (1.0 - p) / Mbar;
    double wlq = b * Ml * p / Mbar;
    if (P->plant & PLANT_SWAP_W) { double t = ws; ws = wlq; wlq = t; }
    double g[3] = {0, 0, 0}, gY[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, gl[3] = {0, 0, 0};
    for (int e = 0; e < P->dim; ++e) {
        if (e == a) {
            g[e] = (W->phi[cR] - W->phi[cL]) / dx;
            gY[e] = (W->Y[cR] - W->Y[cL]) / dx;
            gs[e] = (W->mus[cR] - W->mus[cL]) / dx;
            gl[e] = (W->mul[cR] - W->mul[cL]) / dx;
        } else {
            g[e] = 0.5 * (cgrad(W, W->phi, cL, e, dx) + cgrad(W, W->phi, cR, e, dx));
            gY[e] = 0.5 * (cgrad(W, W->Y, cL, e, dx) + cgrad(W, W->Y, cR, e, dx));
            gs[e] = 0.5 * (cgrad(W, W->mus, cL, e, dx) + cgrad(W, W->mus, cR, e, dx));
            gl[e] = 0.5 * (cgrad(W, W->mul, cL, e, dx) + cgrad(W, W->mul, cR, e, dx));
        }
    }
    double g2 = 0, dY = 0, ds = 0, dl = 0;
    for (int e = 0; e < P->dim; ++e) {
        g2 += g[e] * g[e]; dY += g[e] * gY[e]; ds += g[e] * gs[e]; dl += g[e] * gl[e];
    }
    double r = 1.0 / (g2 + P->delta * P->delta);
    double tsgn = (P->plant & PLANT_TANG_SIGN) ? -1.0 : 1.0;
    double at = (P->plant & PLANT_NO_ANTITRAP) ? 0.0 : 1.0;
    double normal = q * g[a] * dY * r;
    *Fs = normal + Ms * (gs[a] - tsgn * g[a] * ds * r) + at * (1.0 - A) * d * ws * pdot * g[a] * r;
    *Fl = normal + Ml * (gl[a] - tsgn * g[a] * dl * r) - at * (1.0 - A) * d * wlq * pdot * g[a] * r;
    *pf_out = p;
}

static void stage_faces(const orc_params* P, work* W) {
    const layout* L = &W->L;
    for (int a = 0; a < P->dim; ++a) {
        int64_t n0 = W->fn[a][0], n1 = W->fn[a][1], n2 = W->fn[a][2];
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < n2; ++k)
            for (int64_t j = 0; j < n1; ++j)
                for (int64_t i = 0; i < n0; ++i) {
                    /* coordinates of the face's left cell (may be a ghost) */
                    int64_t ci[3] = {i, j, k};
                    ci[a] -= 1;
                    int64_t cL = pidx(L, ci[0], ci[1], ci[2]);
                    int64_t cR = cL + L->s[a];
                    int boundary = (ci[a] == -1) || (ci[a] == L->n[a] - 1);
                    int bc = (ci[a] == -1) ? P->bc_lo[a] : P->bc_hi[a];
                    double Fs = 0.0, Fl = 0.0, pf = 0.0;
                    if (!(boundary && bc == ORC_BC_NOFLUX))
                        face_flux(P, W, cL, cR, a, &Fs, &Fl, &pf);
                    int64_t fi = fidx(W, a, i, j, k);
                    if (P->form == 1) {
                        W->Fa[a][fi] = Fs; W->Fb[a][fi] = Fl;
                    } else {
                        W->Fa[a][fi] = pf * Fs + (1.0 - pf) * Fl;   /* F_c (Eq. model6) */
                        W->Fb[a][fi] = Fs - Fl;                      /* F_d */
                    }
                }
    }
}

/* divergence at interior cell (i,j,k) of the face array pair */
static void divergence(const orc_params* P, const work* W, int64_t i, int64_t j,
                       int64_t k, double* da, double* db) {
    double sa = 0.0, sb = 0.0;
    for (int a = 0; a < P->dim; ++a) {
        int64_t c[3] = {i, j, k};
        int64_t lo = fidx(W, a, c[0], c[1], c[2]);
        c[a] += 1;
        int64_t hi = fidx(W, a, c[0], c[1], c[2]);
        sa += W->Fa[a][hi] - W->Fa[a][lo];
        sb += W->Fb[a][hi] - W->Fb[a][lo];
    }
    *da = sa / P->dx;
    *db = sb / P->dx;
}

static int compute_rates(const orc_params* P, const orc_clock* clk, work* W,
                         const double* phi, const double* cs, const double* cl) {
    stage_fields(P, W, phi, cs, cl);
    stage_phidot(P, clk, W);
    stage_faces(P, W);
    return 0;
}

int orc_rates(const orc_params* P, const orc_clock* clk, const double* phi,
              const double* cs, const double* cl, double* phidot,
              double* cdot, double* ddot) {
    if (!valid_params(P)) return -1;
    work W;
    if (work_alloc(P, &W)) return -1;
    compute_rates(P, clk, &W, phi, cs, cl);
    const layout* L = &W.L;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < L->n[2]; ++k)
        for (int64_t j = 0; j < L->n[1]; ++j)
            for (int64_t i = 0; i < L->n[0]; ++i) {
                int64_t u = uidx(L, i, j, k);
                double da, db;
                divergence(P, &W, i, j, k, &da, &db);
                if (phidot) phidot[u] = W.pd[pidx(L, i, j, k)];
                if (cdot) cdot[u] = da;
                if (ddot) ddot[u] = db;
            }
    work_free(&W);
    return 0;
}

/* ---------------------------------------------------------------- diagnostics */

static double energy_padded(const orc_params* P, const orc_clock* clk, const work* W) {
    const layout* L = &W->L;
    int off[18][3]; double wl[18];
    int m = lap_stencil(P->lap, off, wl);
    double dV = pow(P->dx, P->dim);
    double* part = calloc((size_t)L->n[2] * L->n[1], sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < L->n[2]; ++k)
        for (int64_t j = 0; j < L->n[1]; ++j) {
            double s = 0.0;
            for (int64_t i = 0; i < L->n[0]; ++i) {
                int64_t c = pidx(L, i, j, k);
                double f = W->phi[c], p = W->p[c];
                double theta = theta_at(P, clk, i);
                double bulk = P->H * fdw_of(f) + p * fs_of(P, W->cs[c], theta) +
                              (1.0 - p) * fl_of(W->cl[c]);
                /* gradient energy: (sigma/2) sum over stencil pairs, each pair
                 * once, of w (phi_i - phi_j)^2 / dx^2 */
                double gsum = 0.0;
                for (int e = 0; e < m; ++e) {
                    int64_t o = off[e][0] * L->s[0] + off[e][1] * L->s[1] + off[e][2] * L->s[2];
                    double dphi = W->phi[c + o] - f;
                    gsum += wl[e] * dphi * dphi;
                }
                s += bulk + 0.5 * P->sigma * 0.5 * gsum / (P->dx * P->dx);
            }
            part[k * L->n[1] + j] = s;
        }
    double tot = 0.0;
    for (int64_t r = 0; r < L->n[2] * L->n[1]; ++r) tot += part[r];
    free(part);
    return tot * dV;
}

double orc_energy(const orc_params* P, const orc_clock* clk, const double* phi,
                  const double* cs, const double* cl) {
    if (!valid_params(P)) return NAN;
    work W;
    if (work_alloc(P, &W)) return NAN;
    stage_fields(P, &W, phi, cs, cl);
    double E = energy_padded(P, clk, &W);
    work_free(&W);
    return E;
}

double orc_solute(const orc_params* P, const double* phi, const double* cs,
                  const double* cl) {
    if (!valid_params(P)) return NAN;
    layout L;
    make_layout(P, &L);
    double* part = calloc((size_t)L.n[2] * L.n[1], sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < L.n[2]; ++k)
        for (int64_t j = 0; j < L.n[1]; ++j) {
            double s = 0.0;
            for (int64_t i = 0; i < L.n[0]; ++i) {
                int64_t u = uidx(&L, i, j, k);
                double p = p_of(P, phi[u]);
                s += p * cs[u] + (1.0 - p) * cl[u];   /* Eq. model1 with g = p */
            }
            part[k * L.n[1] + j] = s;
        }
    double tot = 0.0;
    for (int64_t r = 0; r < L.n[2] * L.n[1]; ++r) tot += part[r];
    free(part);
    return tot * pow(P->dx, P->dim);
}

/* Per cell: p(phi) and the mixture c = p c_s + (1 - p) c_l (Eq. model1 with
 * g = p), the terms that orc_solute sums. */
int orc_mixture(const orc_params* P, const double* phi, const double* cs,
                const double* cl, int64_t n, double* p_out, double* c_out) {
    if (!valid_params(P) || n < 0) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t u = 0; u < n; ++u) {
        double p = p_of(P, phi[u]);
        if (p_out) p_out[u] = p;
        if (c_out) c_out[u] = p * cs[u] + (1.0 - p) * cl[u];
    }
    return 0;
}

int orc_front(const orc_params* P, const orc_clock* clk, const double* phi,
              const double* cs, const double* cl, double* x_front, double* c_max) {
    if (!valid_params(P)) return -1;
    layout L;
    make_layout(P, &L);
    double xf = -INFINITY, cm = -INFINITY;
    for (int64_t k = 0; k < L.n[2]; ++k)
        for (int64_t j = 0; j < L.n[1]; ++j) {
            for (int64_t i = L.n[0] - 2; i >= 0; --i) {
                double a = phi[uidx(&L, i, j, k)], b = phi[uidx(&L, i + 1, j, k)];
                if (a >= 0.5 && b < 0.5) {
                    /* linear interpolation between the centres (i + 1/2) dx
                     * and (i + 3/2) dx of the two cells, in the lab frame */
                    double centre = (double)i + 0.5;
                    if (P->plant & PLANT_FRONT_INDEX) centre -= 1.0;
                    if (P->plant & PLANT_FRONT_HALF) centre -= 0.5;
                    double x = (centre + (a - 0.5) / (a - b)) * P->dx +
                               (double)clk->shifts * P->dx;
                    if (x > xf) xf = x;
                    break;
                }
            }
            for (int64_t i = 0; i < L.n[0]; ++i) {
                int64_t u = uidx(&L, i, j, k);
                double p = p_of(P, phi[u]);
                double c = p * cs[u] + (1.0 - p) * cl[u];
                if (c > cm) cm = c;
            }
        }
    *x_front = (xf == -INFINITY) ? NAN : xf;
    *c_max = cm;
    return 0;
}

/* ---------------------------------------------------------------- time step */

int orc_step(const orc_params* P, orc_clock* clk, double* phi, double* cs,
             double* cl, int64_t nsteps, double* energy) {
    if (!valid_params(P) || nsteps < 0) return -1;
    work W;
    if (work_alloc(P, &W)) return -1;
    const layout* L = &W.L;
    int bad = 0;
    for (int64_t s = 0; s < nsteps && !bad; ++s) {
        compute_rates(P, clk, &W, phi, cs, cl);
        if (energy) energy[s] = energy_padded(P, clk, &W);
        double dt = P->dt;
#pragma omp parallel for schedule(static) reduction(| : bad)
        for (int64_t k = 0; k < L->n[2]; ++k)
            for (int64_t j = 0; j < L->n[1]; ++j)
                for (int64_t i = 0; i < L->n[0]; ++i) {
                    int64_t c = pidx(L, i, j, k), u = uidx(L, i, j, k);
                    double da, db;
                    divergence(P, &W, i, j, k, &da, &db);
                    double f = W.phi[c], s_ = W.cs[c], l_ = W.cl[c];
                    double pdot = W.pd[c];
                    double fn = f + dt * pdot;                 /* forward Euler */
                    double csn, cln;
                    if (P->form == 1) {
                        /* literal Eqs. cs_nonvar / cl_nonvar with the sources */
                        double src = -P->A * (s_ - l_) * dp_of(P, f) * pdot;
                        csn = s_ + dt * (da + src);
                        cln = l_ + dt * (db + src);
                    } else {
                        double p = W.p[c];
                        double cc = p * s_ + (1.0 - p) * l_ + dt * da;
                        double dd = (s_ - l_) + dt * db;
                        double pn = p_of(P, fn);
                        csn = cc + (1.0 - pn) * dd;
                        cln = cc - pn * dd;
                    }
                    phi[u] = fn; cs[u] = csn; cl[u] = cln;
                    if (!isfinite(fn) || !isfinite(csn) || !isfinite(cln)) bad |= 1;
                }
        clk->step += 1;
        if (P->shift) {
            double t = (double)clk->step * P->dt;
            /* the window has moved shifts cells when v_pull t first reaches
             * shifts dx (Sec. "Numerical technique") */
            const int64_t ahead = (P->plant & PLANT_SHIFT_EARLY) ? 0 : 1;
            while (P->v_pull * t >= (double)(clk->shifts + ahead) * P->dx) {
                /* cut the cold-end layer, add a fresh hot-end layer */
                int64_t n = L->n[0];
                memmove(phi, phi + 1, (n - 1) * sizeof(double));
                memmove(cs, cs + 1, (n - 1) * sizeof(double));
                memmove(cl, cl + 1, (n - 1) * sizeof(double));
                phi[n - 1] = P->dir_phi; cs[n - 1] = P->dir_cs; cl[n - 1] = P->dir_cl;
                if (P->plant & PLANT_FRESH_CINF) cs[n - 1] = P->c_inf;
                clk->shifts += 1;
            }
        }
    }
    work_free(&W);
    return bad ? -2 : 0;
}
