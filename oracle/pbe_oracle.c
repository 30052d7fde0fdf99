/*
 * Plain FP64 CPU oracle for the explicit high-resolution finite-volume step
 * of the crystallization population balance (Sec. 2.1, Eqs. 1-4; SI Sec. S1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the tests, the smoke check and the CPU baseline of
 * the benchmark do.  It shares no code, header or constant with the CUDA
 * library; it is written for readability, not speed (no blocking, no fusion,
 * each face flux recomputed where it is used).
 *
 * Readings of the paper that the oracle fixes (all also taken by the GPU path):
 *  - semi-discrete (method-of-lines) form of Eq. 3: face flux
 *    F = G (n_upwind + phi(theta) (n_down - n_upwind) / 2), van Leer phi,
 *    advanced in time by two-stage SSP Runge-Kutta (the time accuracy the
 *    (1 - nu) factor of Eq. 3 supplies in the one-step form);
 *  - both directions of the 2-D problem at once (unsplit), with the CFL step
 *    dt = nu / (G1/dL1 + G2/dL2);
 *  - zero ghost cells below L = 0 (two) and above L_max (one): no inflow at
 *    L = 0 except nucleation, free outflow at L_max;
 *  - nucleation B enters the smallest-size cell (1-D) / corner cell (2-D)
 *    as a source B/dL (B/(dL1 dL2)) in every stage;
 *  - the solute balance in the difference form of Eq. 4 after each stage,
 *    with kappa = rho_c k_v times a units factor;
 *  - G = B = 0 whenever S <= 1 (no dissolution).
 * Compile with -ffp-contract=off; IEEE double round-to-nearest.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int ndim;           /* 1 or 2 */
    int n1, n2;         /* cells along L1 (and L2); domain [0, lmax] */
    double lmax1, lmax2;
    int fixed_kinetics; /* 1: G1 = kg1, G2 = kg2, B = kb, independent of S */
    double kg1, g1, kg2, g2, kb, b;
    double cs0, cs1, cs2; /* c*(T) = cs0 + cs1 T + cs2 T^2 */
    double T0, T1, t_cool;
    double kappa;         /* rho_c k_v u */
    double cfl;
} orc_params;

/* ---------------- real instance ---------------- */
typedef struct {
    double dt, C, C1, t, t_new;
    double G1a, G2a, Ba, G1b, G2b, Bb;
    int clipped, out_index;
} steprec_r;
#define SCALAR double
#define SFX(x) x##_r
#define RE(x) (x)
#define SPOW pow
#include "pbe_oracle_core.h"
#undef SCALAR
#undef SFX
#undef RE
#undef SPOW

/* ---------------- complex instance (complex-step derivatives) ---------------- */
typedef struct {
    double complex dt, C, C1, t, t_new;
    double complex G1a, G2a, Ba, G1b, G2b, Bb;
    int clipped, out_index;
} steprec_c;
#define SCALAR double complex
#define SFX(x) x##_c
#define RE(x) creal(x)
#define SPOW cpow
#include "pbe_oracle_core.h"
#undef SCALAR
#undef SFX
#undef RE
#undef SPOW

static size_t ncells(const orc_params* p) { return (size_t)p->n1 * (p->ndim == 2 ? p->n2 : 1); }
static int ncols(const orc_params* p) { return p->ndim == 1 ? 6 : 12; }

static ctx_r make_ctx_r(const orc_params* p)
{
    ctx_r c = {p, p->kg1, p->g1, p->kg2, p->g2, p->kb, p->b};
    return c;
}

/* ------------------------------------------------------------------ */
/* exported entry points                                               */
/* ------------------------------------------------------------------ */

double orc_psi(double a, double b) { return psi_r(a, b); }

double orc_temperature(const orc_params* p, double t) { return temperature_r(p, t); }

void orc_kinetics(const orc_params* p, double C, double t, double* out3)
{
    ctx_r c = make_ctx_r(p);
    kinetics_r(&c, C, t, out3, out3 + 1, out3 + 2);
}

/* out2 = {dt, t_new}; returns 1 if clipped at t_next */
int orc_timestep(const orc_params* p, double G1, double G2, double t, double t_next, double* out2)
{
    ctx_r c = make_ctx_r(p);
    return timestep_r(&c, G1, G2, t, t_next, out2, out2 + 1);
}

void orc_rhs(const orc_params* p, const double* n, double G1, double G2, double B, double* L)
{
    rhs_r(p, n, G1, G2, B, L);
}

/* face fluxes: 1-D F[0..N]; 2-D F1[(N1+1)*N2] (face f, column j at f*N2+j)
 * and F2[N1*(N2+1)] (row i, face f at i*(N2+1)+f) */
void orc_face_fluxes(const orc_params* p, const double* n, double G1, double G2, double* F1, double* F2)
{
    if (p->ndim == 1) {
        for (int f = 0; f <= p->n1; ++f) F1[f] = face1_r(n, p->n1, f, G1);
        return;
    }
    int N1 = p->n1, N2 = p->n2;
    for (int f = 0; f <= N1; ++f)
        for (int j = 0; j < N2; ++j) F1[(size_t)f * N2 + j] = face2_1_r(n, N1, N2, f, j, G1);
    for (int i = 0; i < N1; ++i)
        for (int f = 0; f <= N2; ++f) F2[(size_t)i * (N2 + 1) + f] = face2_2_r(n, N1, N2, i, f, G2);
}

double orc_volume(const orc_params* p, const double* n) { return volume_r(p, n); }

void orc_moments(const orc_params* p, const double* n, double* mu) { moments_r(p, n, mu); }

/* One step; n updated in place; out5 = {dt, C_new, t_new, C1, clipped}. */
void orc_step(const orc_params* p, double* n, double C, double t, double t_next, double* out5)
{
    ctx_r c = make_ctx_r(p);
    double* work = (double*)malloc(3 * ncells(p) * sizeof(double));
    steprec_r rec;
    int clipped = step_r(&c, n, work, &C, &t, t_next, &rec);
    out5[0] = rec.dt; out5[1] = C; out5[2] = t; out5[3] = rec.C1; out5[4] = clipped;
    free(work);
}

/* Full solve. n updated in place to the final state; state_out = {C, t};
 * rows[n_out * ncol].  Returns the number of steps taken. */
long orc_solve(const orc_params* p, double* n, double C, double t,
               const double* t_out, int n_out, double* rows, double* state_out)
{
    ctx_r c = make_ctx_r(p);
    long steps = solve_r(&c, n, &C, &t, t_out, n_out, rows, NULL, NULL, 0);
    state_out[0] = C; state_out[1] = t;
    return steps;
}

/* Complex-step derivative of every output row with respect to one kinetic
 * parameter (index 0..5 = kg1, g1, kg2, g2, kb, b): the parameter is given
 * the imaginary part h and d(row)/d(param) = Im(row) / h.  rows_re gets the
 * real part, drows the derivative.  Returns the number of steps. */
long orc_solve_cs(const orc_params* p, int which, double h, const double* n0, double C0, double t0,
                  const double* t_out, int n_out, double* rows_re, double* drows)
{
    size_t nc = ncells(p);
    int ncol = ncols(p);
    ctx_c c = {p, p->kg1, p->g1, p->kg2, p->g2, p->kb, p->b};
    double complex* slot[6] = {&c.kg1, &c.g1, &c.kg2, &c.g2, &c.kb, &c.b};
    *slot[which] += I * h;
    double complex* n = (double complex*)malloc(nc * sizeof(double complex));
    double complex* rows = (double complex*)malloc((size_t)n_out * ncol * sizeof(double complex));
    for (size_t k = 0; k < nc; ++k) n[k] = n0[k];
    double complex C = C0, t = t0;
    long steps = solve_c(&c, n, &C, &t, t_out, n_out, rows, NULL, NULL, 0);
    for (size_t k = 0; k < (size_t)n_out * ncol; ++k) {
        rows_re[k] = creal(rows[k]);
        drows[k] = cimag(rows[k]) / h;
    }
    free(n); free(rows);
    return steps;
}
