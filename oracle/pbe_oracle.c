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
 * Compile with -ffp-contract=off; IEEE double round-to-nearest.  The
 * element-wise loops of the 2-D right-hand side and of the stage updates of
 * grids of 16384 cells or more may run on several OpenMP threads (for the
 * timed CPU baseline; one thread unless orc_set_threads asks for more); the
 * results are the same on any thread count, since every sum (the moments)
 * runs in one thread in a fixed order.
 */
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif
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
    const double* mlp;    /* learned closure weights (NULL: power law / fixed) */
    int scheme;           /* 0: SSP-RK2 semi-discrete, unsplit; 1: Eq. 3 (one-step high resolution) with
                             Godunov dimensional splitting, dt = cfl * min(dL1/G1, dL2/G2) */
    int growth_form;      /* 0: G = kg s^g; 1: Arrhenius form of Appendix A, G = kg exp(-ea/(T+273.15)) s^g */
    int solubility_form;  /* 0: c* = cs0 + cs1 T + cs2 T^2; 1: c* = cs0 exp(cs1 T) (Appendix A) */
    double ea1, ea2;      /* activation temperatures (K) of the Arrhenius form */
    const double* poly;   /* growth_form 2 (Eq. 6): G_m = sum_{k=1..npoly} poly[m npoly + k - 1] (S - 1)^k,
                             m = 0 (L1) and, in 2-D, 1 (L2) */
    int npoly;
    int mlp_box;          /* learned closure: 1 if its inputs have a training box */
    double mlp_lo[3], mlp_hi[3];
} orc_params;

/* Learned kinetics closure (the empirical hybrid model of Sec. 4.2: a network
 * replaces the growth and nucleation rate expressions inside the solver):
 * a 3 -> 64 -> 64 -> 3 perceptron with SiLU hidden units.  Inputs (fixed
 * affine maps): x0 = 4 (S - 1), x1 = (T - 25) / 10, x2 = 1e-6 V / mu0 with V
 * the volume moment (mu3 in 1-D, mu12 in 2-D).  Outputs: ln G1 = o0 + ln 0.01,
 * ln G2 = o1 + ln 0.005, ln B = o2 + ln 1e5; G = B = 0 for S <= 1.
 * Weight layout: W1[64][3], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]. */
#define MLP_H 64
#define MLP_NW (MLP_H * 3 + MLP_H + MLP_H * MLP_H + MLP_H + 3 * MLP_H + 3)

/* ---------------- real instance ---------------- */
typedef struct {
    double dt, C, C1, t, t_new;
    double G1a, G2a, Ba, G1b, G2b, Bb;
    double r0, r1;  /* moment ratios V/mu0 the closure saw at each stage */
    int clipped, out_index;
} steprec_r;
#define SCALAR double
#define SFX(x) x##_r
#define RE(x) (x)
#define SPOW pow
#define SEXP exp
#include "pbe_oracle_core.h"
#undef SCALAR
#undef SFX
#undef RE
#undef SPOW
#undef SEXP

/* ---------------- complex instance (complex-step derivatives) ---------------- */
typedef struct {
    double complex dt, C, C1, t, t_new;
    double complex G1a, G2a, Ba, G1b, G2b, Bb;
    double complex r0, r1;
    int clipped, out_index;
} steprec_c;
#define SCALAR double complex
#define SFX(x) x##_c
#define RE(x) creal(x)
#define SPOW cpow
#define SEXP cexp
#include "pbe_oracle_core.h"
#undef SCALAR
#undef SFX
#undef RE
#undef SPOW
#undef SEXP

static size_t ncells(const orc_params* p) { return (size_t)p->n1 * (p->ndim == 2 ? p->n2 : 1); }
static int ncols(const orc_params* p) { return p->ndim == 1 ? 6 : 12; }

static ctx_r make_ctx_r(const orc_params* p)
{
    ctx_r c = {p, p->kg1, p->g1, p->kg2, p->g2, p->kb, p->b, p->mlp, p->poly};
    return c;
}

/* ------------------------------------------------------------------ */
/* exported entry points                                               */
/* ------------------------------------------------------------------ */

double orc_psi(double a, double b) { return psi_r(a, b); }

/* Threads of the element-wise loops (the 2-D right-hand side and the stage
 * updates; OpenMP when the library was built with it).  Results do not depend
 * on the count: every sum stays in one thread, in a fixed order.  Returns the
 * count in effect (1 without OpenMP). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

double orc_temperature(const orc_params* p, double t) { return temperature_r(p, t); }

void orc_kinetics(const orc_params* p, double C, double t, double* out3)
{
    ctx_r c = make_ctx_r(p);
    kinetics_r(&c, C, t, 0.0, out3, out3 + 1, out3 + 2);
}

/* learned closure at (C, t) with moment ratio V / mu0 */
void orc_kinetics_mlp(const orc_params* p, double C, double t, double ratio, double* out3)
{
    ctx_r c = make_ctx_r(p);
    kinetics_r(&c, C, t, ratio, out3, out3 + 1, out3 + 2);
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
    double* work = (double*)malloc((3 * ncells(p) + 16) * sizeof(double));
    steprec_r rec;
    int clipped = p->scheme == 1 ? step_lw_r(&c, n, work, &C, &t, t_next, &rec)
                                 : step_r(&c, n, work, &C, &t, t_next, &rec);
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
 * parameter (index 0..5 = kg1, g1, kg2, g2, kb, b; from 6 on, the closure
 * weights or, with growth_form 2, the polynomial coefficients): the parameter
 * is given the imaginary part h and d(row)/d(param) = Im(row) / h.  rows_re
 * gets the real part, drows the derivative.  Returns the number of steps. */
long orc_solve_cs(const orc_params* p, int which, double h, const double* n0, double C0, double t0,
                  const double* t_out, int n_out, double* rows_re, double* drows)
{
    size_t nc = ncells(p);
    int ncol = ncols(p);
    ctx_c c = {p, p->kg1, p->g1, p->kg2, p->g2, p->kb, p->b, NULL, NULL};
    double complex* slot[6] = {&c.kg1, &c.g1, &c.kg2, &c.g2, &c.kb, &c.b};
    double complex* wc = NULL;
    if (p->mlp) {
        wc = (double complex*)malloc(MLP_NW * sizeof(double complex));
        for (int k = 0; k < MLP_NW; ++k) wc[k] = p->mlp[k];
        c.w = wc;
    } else if (p->growth_form == 2) {
        int na = p->npoly * p->ndim;
        wc = (double complex*)malloc((na > 0 ? na : 1) * sizeof(double complex));
        for (int k = 0; k < na; ++k) wc[k] = p->poly[k];
        c.a = wc;
    }
    int nw = p->mlp ? MLP_NW : (p->growth_form == 2 ? p->npoly * p->ndim : 0);
    if (which < 0 || which >= 6 + nw) {
        free(wc);
        return -1;
    }
    if (which < 6) *slot[which] += I * h;
    else wc[which - 6] += I * h;
    double complex* n = (double complex*)malloc(nc * sizeof(double complex));
    double complex* rows = (double complex*)malloc((size_t)n_out * ncol * sizeof(double complex));
    for (size_t k = 0; k < nc; ++k) n[k] = n0[k];
    double complex C = C0, t = t0;
    long steps = solve_c(&c, n, &C, &t, t_out, n_out, rows, NULL, NULL, 0);
    for (size_t k = 0; k < (size_t)n_out * ncol; ++k) {
        rows_re[k] = creal(rows[k]);
        drows[k] = cimag(rows[k]) / h;
    }
    free(n); free(rows); free(wc);
    return steps;
}

/* ------------------------------------------------------------------ */
/* Hand-written discrete adjoint of the step (reverse mode through the  */
/* exact operations of step_r, in reverse order).  Branches follow the  */
/* forward pass: the limiter derivative is that of the branch taken     */
/* (strict same-sign test), S <= 1 has zero derivative, and the step    */
/* length is differentiated through the branch (CFL or output clip)     */
/* that the forward pass took; the number of steps is that of the       */
/* forward pass.                                                        */
/* ------------------------------------------------------------------ */

/* partial derivatives of psi(a, b) = 2ab/(a+b) on its smooth branch.
 * Differences below 2^-959 in magnitude (values far below any physical
 * density, where the ratio b/(a+b) is decided by rounding of underflowing
 * tails) count as flat: derivative 0 (the subgradient convention the GPU
 * adjoint shares). */
#define PSI_FLAT 0x1p-959
static void psi_grad(double a, double b, double* pa, double* pb)
{
    if (((a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0)) && fabs(a) >= PSI_FLAT && fabs(b) >= PSI_FLAT) {
        double qa = b / (a + b), qb = a / (a + b);  /* ratios in (0, 1): no underflow in the tails */
        *pa = 2.0 * qa * qa;
        *pb = 2.0 * qb * qb;
    } else {
        *pa = 0.0;
        *pb = 0.0;
    }
}

/* One line of cells (N cells, element stride st) of D(n)_i = -(h_{i+1} - h_i)/d,
 * h_f = n_{f-1} + psi(n_{f-1} - n_{f-2}, n_f - n_{f-1}) / 2 (zero ghosts).
 * Adds scale * (dD/dn)^T lam to out and returns lam . D(n) = sum_f h_f (lam_f - lam_{f-1}) / d. */
static double line_adjoint(const double* n, const double* lam, int N, long st, double d, double scale, double* out)
{
    double dot = 0.0;
    for (int f = 0; f <= N; ++f) {
        double nm2 = (f - 2 >= 0) ? n[(long)(f - 2) * st] : 0.0;
        double up = (f - 1 >= 0 && f - 1 < N) ? n[(long)(f - 1) * st] : 0.0;
        double dn = (f < N) ? n[(long)f * st] : 0.0;
        double a = up - nm2, b = dn - up;
        double h = up + 0.5 * psi_r(a, b);
        double lamL = (f - 1 >= 0) ? lam[(long)(f - 1) * st] : 0.0;
        double lamR = (f < N) ? lam[(long)f * st] : 0.0;
        double mu = (lamR - lamL) / d;
        dot += h * mu;
        double pa, pb;
        psi_grad(a, b, &pa, &pb);
        if (f - 2 >= 0) out[(long)(f - 2) * st] += scale * mu * (-0.5 * pa);
        if (f - 1 >= 0 && f - 1 < N) out[(long)(f - 1) * st] += scale * mu * (1.0 + 0.5 * (pa - pb));
        if (f < N) out[(long)f * st] += scale * mu * (0.5 * pb);
    }
    return dot;
}

/* out += dt*(G1 dD1/dn + G2 dD2/dn)^T lam; P[0] = lam.D1(n), P[1] = lam.D2(n), P[2] = lam at the inflow cell */
static void stage_adjoint(const orc_params* p, const double* n, const double* lam, double dt, double G1, double G2,
                          double* out, double* P)
{
    P[0] = P[1] = 0.0;
    if (p->ndim == 1) {
        P[0] = line_adjoint(n, lam, p->n1, 1, p->lmax1 / p->n1, dt * G1, out);
    } else {
        int N1 = p->n1, N2 = p->n2;
        double d1 = p->lmax1 / N1, d2 = p->lmax2 / N2;
        for (int j = 0; j < N2; ++j) P[0] += line_adjoint(n + j, lam + j, N1, N2, d1, dt * G1, out + j);
        for (int i = 0; i < N1; ++i)
            P[1] += line_adjoint(n + (size_t)i * N2, lam + (size_t)i * N2, N2, 1, d2, dt * G2, out + (size_t)i * N2);
    }
    P[2] = lam[0];
}

/* weights of the volume moment V = sum w n */
static void volume_weights(const orc_params* p, double* w)
{
    if (p->ndim == 1) {
        double d = p->lmax1 / p->n1;
        for (int i = 0; i < p->n1; ++i) {
            double x = (i + 0.5) * d;
            w[i] = x * x * x * d;
        }
    } else {
        double d1 = p->lmax1 / p->n1, d2 = p->lmax2 / p->n2;
        for (int i = 0; i < p->n1; ++i)
            for (int j = 0; j < p->n2; ++j) {
                double x1 = (i + 0.5) * d1, x2 = (j + 0.5) * d2;
                w[(size_t)i * p->n2 + j] = x1 * x2 * x2 * d1 * d2;
            }
    }
}

/* lam += sum_k seed[k] * (weights of moment k) (output row of the moments) */
static void add_moment_seeds(const orc_params* p, const double* seed, double* lam)
{
    if (p->ndim == 1) {
        double d = p->lmax1 / p->n1;
        for (int i = 0; i < p->n1; ++i) {
            double x = (i + 0.5) * d;
            lam[i] += (seed[0] + seed[1] * x + seed[2] * x * x + seed[3] * x * x * x) * d;
        }
    } else {
        static const int P[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
        static const int Q[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
        double d1 = p->lmax1 / p->n1, d2 = p->lmax2 / p->n2;
        for (int i = 0; i < p->n1; ++i)
            for (int j = 0; j < p->n2; ++j) {
                double x1 = (i + 0.5) * d1, x2 = (j + 0.5) * d2, v = 0.0;
                for (int k = 0; k < 10; ++k) v += seed[k] * pow(x1, P[k]) * pow(x2, Q[k]);
                lam[(size_t)i * p->n2 + j] += v * d1 * d2;
            }
    }
}

/* adjoint of (G1, G2, B) = kinetics(C, t): accumulates into *lC, *lt, lth[6]
 * and, for the polynomial growth law of Eq. 6, lpoly[ndim * npoly] */
static void kinetics_adjoint(const orc_params* p, double C, double t, double lG1, double lG2, double lB,
                             double* lC, double* lt, double* lth, double* lpoly)
{
    if (p->fixed_kinetics) {
        lth[0] += lG1;
        if (p->ndim == 2) lth[2] += lG2;
        lth[4] += lB;
        return;
    }
    double T = temperature_r(p, t);
    double dTdt = (t < p->t_cool) ? (p->T1 - p->T0) / p->t_cool : 0.0;
    double cs = p->cs0 + p->cs1 * T + p->cs2 * T * T;
    double dcs = p->cs1 + 2.0 * p->cs2 * T;
    double s = C / cs - 1.0;
    if (!(s > 0.0)) return;
    double ls = log(s);
    if (p->growth_form == 2) {
        /* G_m = sum_k a_mk s^k: dG_m/da_mk = s^k, dG_m/ds = sum_k k a_mk s^(k-1) */
        double sb = pow(s, p->b), B = p->kb * sb;
        double lsum = lB * p->b * p->kb * pow(s, p->b - 1.0);
        lth[4] += lB * sb;
        lth[5] += lB * B * ls;
        for (int m = 0; m < p->ndim; ++m) {
            const double lG = m == 0 ? lG1 : lG2;
            const double* a = p->poly + (size_t)m * p->npoly;
            double skm1 = 1.0, dG = 0.0;  /* s^(k-1) */
            for (int k = 1; k <= p->npoly; ++k) {
                lpoly[(size_t)m * p->npoly + k - 1] += lG * (skm1 * s);
                dG += k * a[k - 1] * skm1;
                skm1 *= s;
            }
            lsum += lG * dG;
        }
        *lC += lsum / cs;
        *lt += lsum * (-C * dcs / (cs * cs)) * dTdt;
        return;
    }
    double s1 = pow(s, p->g1), sb = pow(s, p->b);
    double G1 = p->kg1 * s1, B = p->kb * sb;
    double lsum = lG1 * p->g1 * p->kg1 * pow(s, p->g1 - 1.0) + lB * p->b * p->kb * pow(s, p->b - 1.0);
    lth[0] += lG1 * s1;
    lth[1] += lG1 * G1 * ls;
    lth[4] += lB * sb;
    lth[5] += lB * B * ls;
    if (p->ndim == 2) {
        double s2 = pow(s, p->g2), G2 = p->kg2 * s2;
        lth[2] += lG2 * s2;
        lth[3] += lG2 * G2 * ls;
        lsum += lG2 * p->g2 * p->kg2 * pow(s, p->g2 - 1.0);
    }
    *lC += lsum / cs;
    *lt += lsum * (-C * dcs / (cs * cs)) * dTdt;
}

static double silu_grad(double z)
{
    double sg = 1.0 / (1.0 + exp(-z));
    return sg * (1.0 + z * (1.0 - sg));
}

/* adjoint of the learned closure at (C, t, ratio): accumulates lC, lt, the
 * adjoint of the moment ratio, and dL/dweights into dW (layout of the weights) */
/* Returns 1, accumulating nothing, when the forward pass took the closure's
 * plain-kinetics fallback at this evaluation (the caller then differentiates
 * the power law); 0 otherwise. */
static int mlp_kinetics_adjoint(const orc_params* p, double C, double t, double ratio, double lG1, double lG2,
                                double lB, double* lC, double* lt, double* lratio, double* dW)
{
    double T = temperature_r(p, t);
    double dTdt = (t < p->t_cool) ? (p->T1 - p->T0) / p->t_cool : 0.0;
    double cs = p->cs0 + p->cs1 * T + p->cs2 * T * T;
    double dcs = p->cs1 + 2.0 * p->cs2 * T;
    double s = C / cs - 1.0;
    if (!(s > 0.0)) return 0;
    const double* w = p->mlp;
    const double* W1 = w;
    const double* b1 = W1 + MLP_H * 3;
    const double* W2 = b1 + MLP_H;
    const double* b2 = W2 + MLP_H * MLP_H;
    const double* W3 = b2 + MLP_H;
    const double* b3 = W3 + 3 * MLP_H;
    double* dW1 = dW;
    double* db1 = dW1 + MLP_H * 3;
    double* dW2 = db1 + MLP_H;
    double* db2 = dW2 + MLP_H * MLP_H;
    double* dW3 = db2 + MLP_H;
    double* db3 = dW3 + 3 * MLP_H;
    double x[3] = {4.0 * s, (T - 25.0) / 10.0, 1e-6 * ratio};
    double z1[MLP_H], a1[MLP_H], z2[MLP_H], a2[MLP_H], o[3];
    for (int h = 0; h < MLP_H; ++h) {
        z1[h] = b1[h] + W1[h * 3] * x[0] + W1[h * 3 + 1] * x[1] + W1[h * 3 + 2] * x[2];
        a1[h] = silu_r(z1[h]);
    }
    for (int h = 0; h < MLP_H; ++h) {
        double z = b2[h];
        for (int j = 0; j < MLP_H; ++j) z += W2[h * MLP_H + j] * a1[j];
        z2[h] = z;
        a2[h] = silu_r(z);
    }
    for (int m = 0; m < 3; ++m) {
        double z = b3[m];
        for (int h = 0; h < MLP_H; ++h) z += W3[m * MLP_H + h] * a2[h];
        o[m] = z;
    }
    const double G[3] = {exp(o[0] + log(0.01)), p->ndim == 2 ? exp(o[1] + log(0.005)) : 0.0, exp(o[2] + log(1e5))};
    if (mlp_fallback_r(p, x, G[0], G[1], G[2])) return 1;
    double lo[3] = {lG1 * G[0], lG2 * G[1], lB * G[2]};
    double la2[MLP_H], lz2[MLP_H], la1[MLP_H], lz1[MLP_H], lx[3] = {0, 0, 0};
    for (int h = 0; h < MLP_H; ++h) la2[h] = 0.0;
    for (int m = 0; m < 3; ++m) {
        db3[m] += lo[m];
        for (int h = 0; h < MLP_H; ++h) {
            dW3[m * MLP_H + h] += lo[m] * a2[h];
            la2[h] += W3[m * MLP_H + h] * lo[m];
        }
    }
    for (int h = 0; h < MLP_H; ++h) lz2[h] = la2[h] * silu_grad(z2[h]);
    for (int j = 0; j < MLP_H; ++j) la1[j] = 0.0;
    for (int h = 0; h < MLP_H; ++h) {
        db2[h] += lz2[h];
        for (int j = 0; j < MLP_H; ++j) {
            dW2[h * MLP_H + j] += lz2[h] * a1[j];
            la1[j] += W2[h * MLP_H + j] * lz2[h];
        }
    }
    for (int h = 0; h < MLP_H; ++h) {
        lz1[h] = la1[h] * silu_grad(z1[h]);
        db1[h] += lz1[h];
        for (int k = 0; k < 3; ++k) {
            dW1[h * 3 + k] += lz1[h] * x[k];
            lx[k] += W1[h * 3 + k] * lz1[h];
        }
    }
    double lS = 4.0 * lx[0];
    double lT = lx[1] / 10.0 - lS * C * dcs / (cs * cs);
    *lC += lS / cs;
    *lt += lT * dTdt;
    *lratio += 1e-6 * lx[2];
    return 0;
}

/* Vector-Jacobian product of a solve.  drows[n_out * ncol]: dL/d(row entries)
 * (the time column is ignored).  Outputs dL/dtheta[6] (kg1, g1, kg2, g2, kb, b),
 * and optionally dL/dn0 (ncell) and dL/dC0; dmlp accumulates dL/d(closure
 * weights), dpoly dL/d(polynomial growth coefficients, growth_form 2; the
 * growth entries of dtheta are then 0).  Returns the number of steps. */
long orc_vjp(const orc_params* p, const double* n0, double C0, double t0, const double* t_out, int n_out,
             const double* drows, double* dtheta, double* dn0, double* dC0, double* dmlp, double* dpoly)
{
    /* adjoint of the SSP-RK2 scheme with the power-law or polynomial growth law only */
    if (p->scheme != 0 || (p->growth_form != 0 && p->growth_form != 2) || p->solubility_form != 0) return -1;
    if (p->growth_form == 2 && (p->mlp || !dpoly)) return -1;
    size_t nc = ncells(p);
    int ncol = ncols(p), nm = ncol - 2;
    double area = (p->ndim == 1) ? p->lmax1 / p->n1 : (p->lmax1 / p->n1) * (p->lmax2 / p->n2);
    double d1 = p->lmax1 / p->n1, d2 = (p->ndim == 2) ? p->lmax2 / p->n2 : 1.0;
    /* forward pass with every step recorded */
    long cap = 1024;
    steprec_r* recs = NULL;
    double* snaps = NULL;
    double* rows = (double*)malloc((size_t)n_out * ncol * sizeof(double));
    double* n = (double*)malloc(nc * sizeof(double));
    long steps;
    for (;;) {
        recs = (steprec_r*)malloc(cap * sizeof(steprec_r));
        snaps = (double*)malloc((size_t)cap * nc * sizeof(double));
        memcpy(n, n0, nc * sizeof(double));
        double C = C0, t = t0;
        ctx_r c = make_ctx_r(p);
        steps = solve_r(&c, n, &C, &t, t_out, n_out, rows, recs, snaps, cap);
        if (steps >= 0) break;
        free(recs); free(snaps);
        cap *= 4;
    }
    double* w = (double*)malloc(nc * sizeof(double));
    double* lam = (double*)calloc(nc, sizeof(double));
    double* lam1 = (double*)malloc(nc * sizeof(double));
    double* lamp = (double*)malloc(nc * sizeof(double));
    double* n1 = (double*)malloc(nc * sizeof(double));
    double* L = (double*)malloc(nc * sizeof(double));
    volume_weights(p, w);
    double lC = 0.0, lt = 0.0;
    double lth[6] = {0, 0, 0, 0, 0, 0};
    for (long k = steps - 1; k >= 0; --k) {
        const steprec_r* r = &recs[k];
        if (r->out_index >= 0) {  /* seeds of the output row emitted at the end of this step */
            const double* sd = drows + (size_t)r->out_index * ncol;
            add_moment_seeds(p, sd + 1, lam);
            lC += sd[1 + nm];
        }
        const double* nk = snaps + (size_t)k * nc;
        rhs_r(p, nk, r->G1a, r->G2a, r->Ba, L);
        for (size_t q = 0; q < nc; ++q) n1[q] = nk[q] + r->dt * L[q];
        /* C' = C - kappa (V' - V0) */
        double lV0 = p->kappa * lC;
        double lCp = lC;
        for (size_t q = 0; q < nc; ++q) lam[q] += -p->kappa * lC * w[q];
        /* n' = n/2 + n2/2 */
        for (size_t q = 0; q < nc; ++q) { lamp[q] = 0.5 * lam[q]; lam[q] = 0.5 * lam[q]; }  /* lam <- lam_n2 */
        /* n2 = n1 + dt L(n1; b) */
        double P[3];
        memcpy(lam1, lam, nc * sizeof(double));
        stage_adjoint(p, n1, lam, r->dt, r->G1b, r->G2b, lam1, P);
        double ldt = r->G1b * P[0] + r->G2b * P[1] + r->Bb * P[2] / area;
        double lG1 = r->dt * P[0], lG2 = r->dt * P[1], lB = r->dt * P[2] / area;
        /* kinetics at (C1, t') */
        double lC1 = 0.0, ltn = lt;
        double lr = 0.0;
        if (p->mlp && !mlp_kinetics_adjoint(p, r->C1, r->t_new, r->r1, lG1, lG2, lB, &lC1, &ltn, &lr, dmlp)) {
            double m0 = mu0_r(p, n1), V1 = volume_r(p, n1);
            for (size_t q = 0; q < nc; ++q) lam1[q] += (lr / m0) * w[q] - (lr * V1 / (m0 * m0)) * area;
        } else {   /* the power law (also the closure's fallback) */
            kinetics_adjoint(p, r->C1, r->t_new, lG1, lG2, lB, &lC1, &ltn, lth, dpoly);
        }
        /* C1 = C - kappa (V1 - V0) */
        lCp += lC1;
        lV0 += p->kappa * lC1;
        for (size_t q = 0; q < nc; ++q) lam1[q] += -p->kappa * lC1 * w[q];
        /* n1 = n + dt L(n; a) */
        for (size_t q = 0; q < nc; ++q) lamp[q] += lam1[q];
        stage_adjoint(p, nk, lam1, r->dt, r->G1a, r->G2a, lamp, P);
        ldt += r->G1a * P[0] + r->G2a * P[1] + r->Ba * P[2] / area;
        lG1 = r->dt * P[0]; lG2 = r->dt * P[1]; lB = r->dt * P[2] / area;
        /* V0 = w . n */
        for (size_t q = 0; q < nc; ++q) lamp[q] += lV0 * w[q];
        /* step length */
        double ltp;
        if (!r->clipped) {
            ltp = ltn;
            ldt += ltn;
            double R = r->G1a / d1 + ((p->ndim == 2) ? r->G2a / d2 : 0.0);
            double dR = -p->cfl / (R * R) * ldt;
            lG1 += dR / d1;
            if (p->ndim == 2) lG2 += dR / d2;
        } else {
            ltp = -ldt;
        }
        /* kinetics at (C, t) */
        lr = 0.0;
        if (p->mlp && !mlp_kinetics_adjoint(p, r->C, r->t, r->r0, lG1, lG2, lB, &lCp, &ltp, &lr, dmlp)) {
            double m0 = mu0_r(p, nk), V0 = volume_r(p, nk);
            for (size_t q = 0; q < nc; ++q) lamp[q] += (lr / m0) * w[q] - (lr * V0 / (m0 * m0)) * area;
        } else {   /* the power law (also the closure's fallback) */
            kinetics_adjoint(p, r->C, r->t, lG1, lG2, lB, &lCp, &ltp, lth, dpoly);
        }
        memcpy(lam, lamp, nc * sizeof(double));
        lC = lCp;
        lt = ltp;
    }
    if (n_out > 0 && t_out[0] == t0) {  /* row emitted from the initial state */
        add_moment_seeds(p, drows + 1, lam);
        lC += drows[1 + nm];
    }
    for (int q = 0; q < 6; ++q) dtheta[q] = lth[q];
    if (dn0) memcpy(dn0, lam, nc * sizeof(double));
    if (dC0) *dC0 = lC;
    free(recs); free(snaps); free(rows); free(n); free(w); free(lam); free(lam1); free(lamp); free(n1); free(L);
    return steps;
}
