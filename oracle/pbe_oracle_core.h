/*
 * Scalar-generic body of the CPU oracle.  Included twice by pbe_oracle.c:
 * once with SCALAR = double (the oracle proper) and once with
 * SCALAR = double complex (complex-step differentiation of the same
 * arithmetic, used only to pin the hand-written adjoint).
 *
 * Macros expected from the includer:
 *   SCALAR   element type
 *   SFX(x)   name mangling (x##_r or x##_c)
 *   RE(x)    real part used for every branch decision
 *   SPOW     power function for SCALAR
 *
 * Test infrastructure only: nothing in the product path includes this.
 */

/* van Leer limited slope phi(theta) * b at one face.
 * Supporting Information Sec. S1.1: theta = (f_{i} - f_{i-1}) / (f_{i+1} - f_{i})
 * (the smoothness ratio, shifted to face i+1/2) and
 * phi(theta) = (theta + |theta|) / (1 + |theta|).
 * With a = f_i - f_{i-1} and b = f_{i+1} - f_i, phi(a/b) * b equals
 * 2ab/(a+b) when a and b have the same strict sign and 0 otherwise; this
 * form is evaluated so that b = 0 gives the limit 0 instead of 0 * inf. */
static SCALAR SFX(psi)(SCALAR a, SCALAR b)
{
    if ((RE(a) > 0.0 && RE(b) > 0.0) || (RE(a) < 0.0 && RE(b) < 0.0))
        return 2.0 * a * (b / (a + b));
    return 0.0;
}

typedef struct {
    const orc_params* p;
    SCALAR kg1, g1, kg2, g2, kb, b; /* kinetic parameters (differentiable) */
    const SCALAR* w;                /* learned closure weights, NULL unless p->mlp */
    const SCALAR* a;                /* polynomial growth coefficients (growth_form 2, differentiable) */
} SFX(ctx);

static SCALAR SFX(silu)(SCALAR z) { return z / (1.0 + SEXP(-z)); }

/* the closure's perceptron: o = W3 silu(W2 silu(W1 x + b1) + b2) + b3 */
static void SFX(mlp_forward)(const SCALAR* w, const SCALAR* x, SCALAR* o)
{
    const SCALAR* W1 = w;
    const SCALAR* b1 = W1 + MLP_H * 3;
    const SCALAR* W2 = b1 + MLP_H;
    const SCALAR* b2 = W2 + MLP_H * MLP_H;
    const SCALAR* W3 = b2 + MLP_H;
    const SCALAR* b3 = W3 + 3 * MLP_H;
    SCALAR a1[MLP_H], a2[MLP_H];
    for (int h = 0; h < MLP_H; ++h)
        a1[h] = SFX(silu)(b1[h] + W1[h * 3] * x[0] + W1[h * 3 + 1] * x[1] + W1[h * 3 + 2] * x[2]);
    for (int h = 0; h < MLP_H; ++h) {
        SCALAR z = b2[h];
        for (int j = 0; j < MLP_H; ++j) z = z + W2[h * MLP_H + j] * a1[j];
        a2[h] = SFX(silu)(z);
    }
    for (int m = 0; m < 3; ++m) {
        SCALAR z = b3[m];
        for (int h = 0; h < MLP_H; ++h) z = z + W3[m * MLP_H + h] * a2[h];
        o[m] = z;
    }
}

/* Temperature of the linear cooling profile at time t. */
static SCALAR SFX(temperature)(const orc_params* p, SCALAR t)
{
    SCALAR frac = (RE(t) < p->t_cool) ? t / p->t_cool : (SCALAR)1.0;
    return p->T0 + (p->T1 - p->T0) * frac;
}

/* Solubility: polynomial, or the exponential c* = a exp(b T) of Appendix A. */
static SCALAR SFX(solubility)(const orc_params* p, SCALAR T)
{
    if (p->solubility_form == 1) return p->cs0 * SEXP(p->cs1 * T);
    return p->cs0 + p->cs1 * T + p->cs2 * T * T;
}

/* The closure's plain-kinetics fallback (its rates stay those of the power
 * law of the kinetic parameters, which remain the judge of the closure): taken
 * when an input leaves the training box (if one is set) or a rate is not
 * finite.  The box test is on the FP64 inputs, as on the GPU. */
static int SFX(mlp_fallback)(const orc_params* p, const SCALAR* x, SCALAR G1, SCALAR G2, SCALAR B)
{
    if (p->mlp_box)
        for (int k = 0; k < 3; ++k)
            if (!(RE(x[k]) >= p->mlp_lo[k] && RE(x[k]) <= p->mlp_hi[k])) return 1;
    return !(isfinite(RE(G1)) && isfinite(RE(G2)) && isfinite(RE(B)));
}

/* Kinetics at concentration C and time t.
 * S = c / c*(T) (Sec. 2.1); growth and nucleation only for S > 1
 * (Appendix A: growth "only applies when S exceeds one").
 * G_m = kg_m (S-1)^g_m, B = kb (S-1)^b. */
static void SFX(kinetics)(const SFX(ctx)* c, SCALAR C, SCALAR t, SCALAR ratio,
                          SCALAR* G1, SCALAR* G2, SCALAR* B)
{
    const orc_params* p = c->p;
    if (c->w) {  /* learned closure */
        SCALAR T = SFX(temperature)(p, t);
        SCALAR csat = SFX(solubility)(p, T);
        SCALAR s = C / csat - 1.0;
        if (!(RE(s) > 0.0)) {
            *G1 = 0.0; *G2 = 0.0; *B = 0.0;
            return;
        }
        SCALAR x[3] = {4.0 * s, (T - 25.0) / 10.0, 1e-6 * ratio};
        SCALAR o[3];
        SFX(mlp_forward)(c->w, x, o);
        *G1 = SEXP(o[0] + log(0.01));
        *G2 = (p->ndim == 2) ? SEXP(o[1] + log(0.005)) : (SCALAR)0.0;
        *B = SEXP(o[2] + log(1e5));
        if (!SFX(mlp_fallback)(p, x, *G1, *G2, *B)) return;
        /* else: the power law below */
    }
    if (p->fixed_kinetics) {
        *G1 = c->kg1;
        *G2 = (p->ndim == 2) ? c->kg2 : (SCALAR)0.0;
        *B = c->kb;
        return;
    }
    SCALAR T = SFX(temperature)(p, t);
    SCALAR csat = SFX(solubility)(p, T);
    SCALAR s = C / csat - 1.0;
    if (!(RE(s) > 0.0)) {
        *G1 = 0.0; *G2 = 0.0; *B = 0.0;
        return;
    }
    if (p->growth_form == 2) {  /* Eq. 6: G_m = a_m1 (S-1) + a_m2 (S-1)^2 + ... + a_mK (S-1)^K */
        SCALAR G[2] = {0.0, 0.0};
        for (int m = 0; m < p->ndim; ++m) {
            SCALAR sk = s;  /* (S-1)^k */
            for (int k = 1; k <= p->npoly; ++k) {
                G[m] += c->a[m * p->npoly + k - 1] * sk;
                sk *= s;
            }
        }
        *G1 = G[0];
        *G2 = G[1];
        *B = c->kb * SPOW(s, c->b);
        return;
    }
    SCALAR a1 = 1.0, a2 = 1.0;
    if (p->growth_form == 1) {  /* Appendix A: kg exp(-kg2 / (T + 273.15)) (S - 1)^kg3 */
        a1 = SEXP(-p->ea1 / (T + 273.15));
        a2 = SEXP(-p->ea2 / (T + 273.15));
    }
    *G1 = c->kg1 * a1 * SPOW(s, c->g1);
    *G2 = (p->ndim == 2) ? c->kg2 * a2 * SPOW(s, c->g2) : (SCALAR)0.0;
    *B = c->kb * SPOW(s, c->b);
}

/* CFL time step (Sec. 2.1 and SI Sec. S1.1), clipped at the next output
 * time.  dt_cfl = nu / (G1/dL1 + G2/dL2); the step is clipped when
 * dt_cfl is not strictly smaller than t_next - t.  Returns 1 if clipped. */
static int SFX(timestep)(const SFX(ctx)* c, SCALAR G1, SCALAR G2, SCALAR t,
                         double t_next, SCALAR* dt, SCALAR* t_new)
{
    const orc_params* p = c->p;
    double d1 = p->lmax1 / p->n1;
    SCALAR rate = G1 / d1;
    if (p->ndim == 2) {
        SCALAR r2 = G2 / (p->lmax2 / p->n2);
        if (p->scheme == 1) {  /* SI Sec. S1.1: dt = nu min(dL1/G1, dL2/G2) */
            if (RE(r2) > RE(rate)) rate = r2;
        } else {
            rate = rate + r2;
        }
    }
    SCALAR rem = t_next - t;
    if (RE(rate) > 0.0) {
        SCALAR dtc = p->cfl / rate;
        if (RE(dtc) < RE(rem)) {
            *dt = dtc;
            *t_new = t + dtc;
            return 0;
        }
    }
    *dt = rem;
    *t_new = t_next;
    return 1;
}

/* value of the distribution with zero ghost cells outside [0, N) */
static SCALAR SFX(at1)(const SCALAR* n, int N, int i)
{
    return (i < 0 || i >= N) ? (SCALAR)0.0 : n[i];
}

/* Growth flux through face f of a 1-D grid (face f lies between cells
 * f-1 and f; growth is positive so the upwind cell is f-1):
 * F_f = G (n_{f-1} + phi * (n_f - n_{f-1}) / 2)   (Eq. 3, flux form). */
static SCALAR SFX(face1)(const SCALAR* n, int N, int f, SCALAR G)
{
    SCALAR nm2 = SFX(at1)(n, N, f - 2), nm1 = SFX(at1)(n, N, f - 1), n0 = SFX(at1)(n, N, f);
    return G * (nm1 + 0.5 * SFX(psi)(nm1 - nm2, n0 - nm1));
}

/* Right-hand side L(n) of the semi-discrete 1-D PBE:
 * L_i = -(F_{i+1/2} - F_{i-1/2}) / dL, plus the nucleation inflow B/dL
 * into the smallest-size cell. */
static void SFX(rhs1)(const orc_params* p, const SCALAR* n, SCALAR G, SCALAR B, SCALAR* L)
{
    int N = p->n1;
    double d = p->lmax1 / N;
    for (int i = 0; i < N; ++i)
        L[i] = -(SFX(face1)(n, N, i + 1, G) - SFX(face1)(n, N, i, G)) / d;
    L[0] = L[0] + B / d;
}

/* 2-D distribution n[i*N2 + j]: i indexes L1, j indexes L2. */
static SCALAR SFX(at2)(const SCALAR* n, int N1, int N2, int i, int j)
{
    return (i < 0 || i >= N1 || j < 0 || j >= N2) ? (SCALAR)0.0 : n[(size_t)i * N2 + j];
}

/* flux along L1 through the face between cells (f-1, j) and (f, j) */
static SCALAR SFX(face2_1)(const SCALAR* n, int N1, int N2, int f, int j, SCALAR G1)
{
    SCALAR nm2 = SFX(at2)(n, N1, N2, f - 2, j), nm1 = SFX(at2)(n, N1, N2, f - 1, j),
           n0 = SFX(at2)(n, N1, N2, f, j);
    return G1 * (nm1 + 0.5 * SFX(psi)(nm1 - nm2, n0 - nm1));
}

/* flux along L2 through the face between cells (i, f-1) and (i, f) */
static SCALAR SFX(face2_2)(const SCALAR* n, int N1, int N2, int i, int f, SCALAR G2)
{
    SCALAR nm2 = SFX(at2)(n, N1, N2, i, f - 2), nm1 = SFX(at2)(n, N1, N2, i, f - 1),
           n0 = SFX(at2)(n, N1, N2, i, f);
    return G2 * (nm1 + 0.5 * SFX(psi)(nm1 - nm2, n0 - nm1));
}

/* Right-hand side of the 2-D PBE (Eq. 1), both directions at once
 * (unsplit), nucleation inflow B/(dL1 dL2) into the corner cell (0,0). */
static void SFX(rhs2)(const orc_params* p, const SCALAR* n, SCALAR G1, SCALAR G2, SCALAR B, SCALAR* L)
{
    int N1 = p->n1, N2 = p->n2;
    double d1 = p->lmax1 / N1, d2 = p->lmax2 / N2;
    /* every L[i][j] is computed on its own: the rows may run on several threads */
#pragma omp parallel for schedule(static) if ((long)N1 * N2 >= 16384)
    for (int i = 0; i < N1; ++i)
        for (int j = 0; j < N2; ++j) {
            SCALAR dF1 = SFX(face2_1)(n, N1, N2, i + 1, j, G1) - SFX(face2_1)(n, N1, N2, i, j, G1);
            SCALAR dF2 = SFX(face2_2)(n, N1, N2, i, j + 1, G2) - SFX(face2_2)(n, N1, N2, i, j, G2);
            L[(size_t)i * N2 + j] = -dF1 / d1 - dF2 / d2;
        }
    L[0] = L[0] + B / (d1 * d2);
}

static void SFX(rhs)(const orc_params* p, const SCALAR* n, SCALAR G1, SCALAR G2, SCALAR B, SCALAR* L)
{
    if (p->ndim == 1) SFX(rhs1)(p, n, G1, B, L);
    else SFX(rhs2)(p, n, G1, G2, B, L);
}

/* zeroth moment mu0 = sum n dA */
static SCALAR SFX(mu0)(const orc_params* p, const SCALAR* n)
{
    SCALAR v = 0.0;
    size_t nc = (size_t)p->n1 * (p->ndim == 2 ? p->n2 : 1);
    double dA = (p->ndim == 1) ? p->lmax1 / p->n1 : (p->lmax1 / p->n1) * (p->lmax2 / p->n2);
    for (size_t k = 0; k < nc; ++k) v = v + n[k] * dA;
    return v;
}

/* Crystal volume integral of Eq. 2 by the midpoint rule at cell centres
 * x_i = (i + 1/2) dL:  1-D  mu3 = sum x^3 n dL;  2-D  mu12 = sum x1 x2^2 n dL1 dL2. */
static SCALAR SFX(volume)(const orc_params* p, const SCALAR* n)
{
    SCALAR v = 0.0;
    if (p->ndim == 1) {
        double d = p->lmax1 / p->n1;
        for (int i = 0; i < p->n1; ++i) {
            double x = (i + 0.5) * d;
            v = v + x * x * x * n[i] * d;
        }
    } else {
        double d1 = p->lmax1 / p->n1, d2 = p->lmax2 / p->n2;
        for (int i = 0; i < p->n1; ++i) {
            double x1 = (i + 0.5) * d1;
            for (int j = 0; j < p->n2; ++j) {
                double x2 = (j + 0.5) * d2;
                v = v + x1 * x2 * x2 * n[(size_t)i * p->n2 + j] * d1 * d2;
            }
        }
    }
    return v;
}

/* Moments (SI Eq. for mu_pq) by the midpoint rule.  1-D: mu0..mu3.
 * 2-D: mu00, mu10, mu01, mu20, mu11, mu02, mu30, mu21, mu12, mu03. */
static void SFX(moments)(const orc_params* p, const SCALAR* n, SCALAR* mu)
{
    if (p->ndim == 1) {
        double d = p->lmax1 / p->n1;
        for (int k = 0; k < 4; ++k) mu[k] = 0.0;
        for (int i = 0; i < p->n1; ++i) {
            double x = (i + 0.5) * d;
            mu[0] = mu[0] + n[i] * d;
            mu[1] = mu[1] + x * n[i] * d;
            mu[2] = mu[2] + x * x * n[i] * d;
            mu[3] = mu[3] + x * x * x * n[i] * d;
        }
    } else {
        static const int P[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
        static const int Q[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
        double d1 = p->lmax1 / p->n1, d2 = p->lmax2 / p->n2;
        for (int k = 0; k < 10; ++k) mu[k] = 0.0;
        for (int i = 0; i < p->n1; ++i) {
            double x1 = (i + 0.5) * d1;
            for (int j = 0; j < p->n2; ++j) {
                double x2 = (j + 0.5) * d2;
                SCALAR v = n[(size_t)i * p->n2 + j] * d1 * d2;
                for (int k = 0; k < 10; ++k)
                    mu[k] = mu[k] + pow(x1, P[k]) * pow(x2, Q[k]) * v;
            }
        }
    }
}

/* One SSP-RK2 step of the semi-discrete PBE with the discrete solute
 * balance of Eq. 4 applied after each stage.
 * State (n, C, t) -> (n_new, C_new, t_new); work holds 3 * ncell.
 * Per-step scalars are written to rec when it is non-NULL. */
static int SFX(step)(const SFX(ctx)* c, SCALAR* n, SCALAR* work, SCALAR* C, SCALAR* t,
                     double t_next, SFX(steprec)* rec)
{
    const orc_params* p = c->p;
    size_t nc = (size_t)p->n1 * (p->ndim == 2 ? p->n2 : 1);
    SCALAR* L = work;
    SCALAR* n1 = work + nc;
    SCALAR G1a, G2a, Ba, G1b, G2b, Bb, dt, t_new;

    /* kinetics and time step from the state at the start of the step */
    SCALAR V0 = SFX(volume)(p, n);
    SCALAR r0 = c->w ? V0 / SFX(mu0)(p, n) : (SCALAR)0.0;
    SFX(kinetics)(c, *C, *t, r0, &G1a, &G2a, &Ba);
    int clipped = SFX(timestep)(c, G1a, G2a, *t, t_next, &dt, &t_new);

    /* stage 1: n1 = n + dt L(n); solute balance C1 = C - kappa (V(n1) - V(n)) */
    SFX(rhs)(p, n, G1a, G2a, Ba, L);
#pragma omp parallel for schedule(static) if (nc >= 16384)
    for (size_t k = 0; k < nc; ++k) n1[k] = n[k] + dt * L[k];
    SCALAR V1 = SFX(volume)(p, n1);
    SCALAR C1 = *C - p->kappa * (V1 - V0);
    SCALAR r1 = c->w ? V1 / SFX(mu0)(p, n1) : (SCALAR)0.0;

    /* stage 2 with kinetics at (C1, t + dt); n_new = n/2 + (n1 + dt L(n1))/2 */
    SFX(kinetics)(c, C1, t_new, r1, &G1b, &G2b, &Bb);
    SFX(rhs)(p, n1, G1b, G2b, Bb, L);
#pragma omp parallel for schedule(static) if (nc >= 16384)
    for (size_t k = 0; k < nc; ++k) n[k] = 0.5 * n[k] + 0.5 * (n1[k] + dt * L[k]);
    SCALAR C_new = *C - p->kappa * (SFX(volume)(p, n) - V0);

    if (rec) {
        rec->dt = dt; rec->C = *C; rec->C1 = C1; rec->t = *t; rec->t_new = t_new;
        rec->G1a = G1a; rec->G2a = G2a; rec->Ba = Ba;
        rec->G1b = G1b; rec->G2b = G2b; rec->Bb = Bb;
        rec->clipped = clipped;
        rec->r0 = r0; rec->r1 = r1;
    }
    *C = C_new;
    *t = t_new;
    return clipped;
}

/* One sweep of Eq. 3 along a line of N cells with element stride st:
 * f_i <- f_i - nu (f_i - f_{i-1})
 *        - nu (1 - nu) / 2 [phi_{i+1/2} (f_{i+1} - f_i) - phi_{i-1/2} (f_i - f_{i-1})],
 * phi the van Leer limiter of the smoothness ratio (SI Sec. S1.1), zero
 * ghost cells; line is overwritten, tmp holds N values. */
static void SFX(lw_line)(SCALAR* line, long st, int N, SCALAR nu, SCALAR* tmp)
{
    for (int i = 0; i < N; ++i) {
        SCALAR fm2 = (i - 2 >= 0) ? line[(long)(i - 2) * st] : (SCALAR)0.0;
        SCALAR fm1 = (i - 1 >= 0) ? line[(long)(i - 1) * st] : (SCALAR)0.0;
        SCALAR f0 = line[(long)i * st];
        SCALAR fp1 = (i + 1 < N) ? line[(long)(i + 1) * st] : (SCALAR)0.0;
        SCALAR lim_p = SFX(psi)(f0 - fm1, fp1 - f0);    /* phi_{i+1/2} (f_{i+1} - f_i) */
        SCALAR lim_m = SFX(psi)(fm1 - fm2, f0 - fm1);   /* phi_{i-1/2} (f_i - f_{i-1}) */
        tmp[i] = f0 - nu * (f0 - fm1) - 0.5 * nu * (1.0 - nu) * (lim_p - lim_m);
    }
    for (int i = 0; i < N; ++i) line[(long)i * st] = tmp[i];
}

/* One time step of the paper's scheme: Eq. 3 along L1, then along L2
 * (Godunov splitting, Sec. 2.1), nucleation inflow B dt / dA into the
 * smallest-size cell, then the solute balance of Eq. 4. */
static int SFX(step_lw)(const SFX(ctx)* c, SCALAR* n, SCALAR* work, SCALAR* C, SCALAR* t, double t_next,
                        SFX(steprec)* rec)
{
    const orc_params* p = c->p;
    SCALAR G1, G2, B, dt, t_new;
    SCALAR V0 = SFX(volume)(p, n);
    SCALAR r0 = c->w ? V0 / SFX(mu0)(p, n) : (SCALAR)0.0;
    SFX(kinetics)(c, *C, *t, r0, &G1, &G2, &B);
    int clipped = SFX(timestep)(c, G1, G2, *t, t_next, &dt, &t_new);
    double d1 = p->lmax1 / p->n1;
    if (p->ndim == 1) {
        SFX(lw_line)(n, 1, p->n1, G1 * dt / d1, work);
        n[0] = n[0] + B * dt / d1;
    } else {
        int N1 = p->n1, N2 = p->n2;
        double d2 = p->lmax2 / N2;
        for (int j = 0; j < N2; ++j) SFX(lw_line)(n + j, N2, N1, G1 * dt / d1, work);
        for (int i = 0; i < N1; ++i) SFX(lw_line)(n + (size_t)i * N2, 1, N2, G2 * dt / d2, work);
        n[0] = n[0] + B * dt / (d1 * d2);
    }
    SCALAR C_new = *C - p->kappa * (SFX(volume)(p, n) - V0);
    if (rec) {
        rec->dt = dt; rec->C = *C; rec->C1 = *C; rec->t = *t; rec->t_new = t_new;
        rec->G1a = G1; rec->G2a = G2; rec->Ba = B;
        rec->G1b = 0.0; rec->G2b = 0.0; rec->Bb = 0.0;
        rec->clipped = clipped;
        rec->r0 = r0; rec->r1 = 0.0;
    }
    *C = C_new;
    *t = t_new;
    return clipped;
}

/* Output row: t, moments, C. */
static void SFX(emit)(const orc_params* p, const SCALAR* n, SCALAR C, SCALAR t, SCALAR* row)
{
    int nm = (p->ndim == 1) ? 4 : 10;
    row[0] = t;
    SFX(moments)(p, n, row + 1);
    row[1 + nm] = C;
}

/* March from (n, C, t) through the increasing output times t_out[0..n_out),
 * landing on each exactly (Fig. 1 loop).  An output time equal to the
 * current time emits the current state without stepping. */
static long SFX(solve)(const SFX(ctx)* c, SCALAR* n, SCALAR* C, SCALAR* t,
                       const double* t_out, int n_out, SCALAR* rows,
                       SFX(steprec)* recs, SCALAR* snaps, long max_recs)
{
    const orc_params* p = c->p;
    size_t nc = (size_t)p->n1 * (p->ndim == 2 ? p->n2 : 1);
    int ncol = (p->ndim == 1) ? 6 : 12;
    SCALAR* work = (SCALAR*)malloc((3 * nc + 16) * sizeof(SCALAR));
    long steps = 0;
    for (int j = 0; j < n_out; ++j) {
        while (RE(*t) < t_out[j]) {
            if (recs && steps >= max_recs) { free(work); return -1; }
            if (snaps) memcpy(snaps + (size_t)steps * nc, n, nc * sizeof(SCALAR));
            if (p->scheme == 1)
                SFX(step_lw)(c, n, work, C, t, t_out[j], recs ? recs + steps : NULL);
            else
                SFX(step)(c, n, work, C, t, t_out[j], recs ? recs + steps : NULL);
            if (recs) recs[steps].out_index = -1;
            ++steps;
        }
        if (recs && steps > 0 && RE(*t) == t_out[j]) recs[steps - 1].out_index = j;
        SFX(emit)(p, n, *C, *t, rows + (size_t)j * ncol);
    }
    free(work);
    return steps;
}
