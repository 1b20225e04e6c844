/*
 * dirac_oracle.c -- plain FP64 CPU oracle for the split-operator solution of
 * the momentum-space massless Dirac equation (arXiv 1607.03062).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code, header,
 * table or constant generator with the CUDA library; it is written to be
 * checked against the paper's equations by eye, not to be fast.
 *
 * Units: hbar = v_F = e = 1, energies and momenta in eV, time in hbar/eV.
 *
 * What it computes, in the paper's order:
 *   Sec. II, Eq. (dirac_eq_mom):  i d/dt psi = +/- sigma.(p + A(t)) psi   (valley K+/K-)
 *   Sec. II, Eq. (free_spin1..4): adiabatic free spinors u (positive energy)
 *                                 and v (negative energy), normalised here to 1
 *   Sec. III, Eq. (ev_op_dt):     U(t_f,t_i) = product of N one-step operators
 *   Sec. III, Eq. (approx_time):  one step = exp{-/+ i dt sigma.P(t_{n+1/2})}, P at
 *                                 the midpoint of the step
 *   Sec. III, closed form after Eq. (approx_time):
 *                                 exp = I cos(dt E) - i (sigma.P / E) sin(dt E)
 *   Sec. II, Eq. (pair_prod_homo): |c+|^2 = |u_out^dag psi(t_f)|^2, and the pair
 *                                 density n = 4/(2 pi)^2 * sum |c+|^2 hx hy
 *                                 (factor 4: spin s = +/-1 times valleys K+/-).
 *
 * Readings of the paper that are taken here (each listed in the design notes):
 *   - the initial state of the point p is the negative-energy spinor of
 *     sigma.(p + A_in) (the paper labels it v(t,-p) but writes it with p + eA);
 *   - the step covering [t_i + n dt, t_i + (n+1) dt] uses A at its own midpoint;
 *   - the grid is cell centred: p_i = p_min + (i + 1/2) h.
 *
 * The "STRANG_XY" scheme is not in the paper: it splits sigma.P into its
 * sigma_x and sigma_y parts, e^{-i dt/2 Px sx} e^{-i dt Py sy} e^{-i dt/2 Px sx},
 * each factor a closed-form rotation.  Here it is applied unmerged.
 *
 * The "MAGNUS4" scheme is the higher-order decomposition Sec. III says the
 * midpoint rule can be improved to: the fourth-order Magnus integrator with two
 * Gauss points per step, t_n + (1/2 -/+ sqrt(3)/6) dt:
 *   Omega = dt/2 (A1 + A2) - sqrt(3) dt^2 / 12 [A1, A2],  A_k = -i valley sigma.P_k,
 *   U_n = exp(Omega).
 * Here Omega is formed as a 2x2 matrix from that definition, and its
 * exponential is taken in closed form (Omega is traceless anti-Hermitian).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* Pulse models (the workload).  A(t) is the vector potential in eV (e = 1).  */
/* ------------------------------------------------------------------------- */

enum {
    ORC_PULSE_ZERO = 0,        /* A = 0 on [0, T]                                   */
    ORC_PULSE_SIN2 = 1,        /* (E0/w) sin^2(pi t/T) (sin wt, eps cos wt)          */
    ORC_PULSE_GAUSS = 2,       /* (E0/w) exp(-(t-t0)^2/tau^2) (sin wt, eps cos wt)   */
    ORC_PULSE_TWO_COLOUR = 3,  /* sin^2 envelope, colours w and 2w                   */
    ORC_PULSE_CONST_FIELD = 4, /* A_x = -E0 (t - T/2): constant field E_x = E0       */
    ORC_PULSE_PAPER = 5        /* Sec. IV, Eq. (elec_field), A_x = -int E_x dt       */
};

typedef struct {
    int32_t kind;
    int32_t pad;
    double E0;      /* field amplitude, eV^2                                  */
    double omega;   /* carrier angular frequency, eV                          */
    double T;       /* pulse duration t_f - t_i (t_i = 0)                     */
    double tau;     /* Gaussian width                                         */
    double t0;      /* Gaussian centre                                        */
    double eps;     /* ellipticity (y amplitude / x amplitude)                */
    double phase2;  /* two-colour: phase of the 2w colour                     */
    double Omega_rise; /* paper pulse envelope frequencies                    */
    double Omega_fall;
    double phi;     /* paper pulse envelope (carrier) phase                   */
} orc_pulse;

/* Paper pulse, Sec. IV Eq. (elec_field), with the reading that the fall factor
 * is cos^2(Omega_fall (t - t_f + pi/(2 Omega_fall))) so that the envelope is
 * continuous and falls to zero at t_f. */
static double paper_field_x(const orc_pulse *s, double t)
{
    double env;
    double rise_end = M_PI / (2.0 * s->Omega_rise);
    double fall_start = s->T - M_PI / (2.0 * s->Omega_fall);
    if (t < 0.0 || t > s->T)
        return 0.0;
    if (t < rise_end) {
        double sr = sin(s->Omega_rise * t);
        env = sr * sr;
    } else if (t > fall_start) {
        double cf = cos(s->Omega_fall * (t - fall_start));
        env = cf * cf;
    } else {
        env = 1.0;
    }
    return s->E0 * env * cos(s->omega * t + s->phi);
}

/* A_x(t) = -int_0^t E_x for the paper pulse, by composite 8-point
 * Gauss-Legendre quadrature on panels of length at most 1/(4 omega).  Plain and
 * slow; exact to rounding for the smooth pieces. */
static double paper_A_x(const orc_pulse *s, double t)
{
    static const double x8[4] = {0.1834346424956498, 0.5255324099163290,
                                 0.7966664774136267, 0.9602898564975363};
    static const double w8[4] = {0.3626837833783620, 0.3137066458778873,
                                 0.2223810344533745, 0.1012285362903763};
    double breaks[4];
    double acc = 0.0;
    int nb = 0, k;
    double a = 0.0;
    if (t <= 0.0)
        return 0.0;
    if (t > s->T)
        t = s->T;
    /* split at the envelope's kinks so each panel is smooth */
    breaks[nb++] = M_PI / (2.0 * s->Omega_rise);
    breaks[nb++] = s->T - M_PI / (2.0 * s->Omega_fall);
    breaks[nb++] = t;
    for (k = 0; k < nb; ++k) {
        double b = breaks[k] < t ? breaks[k] : t;
        if (b <= a)
            continue;
        {
            double len = b - a;
            double hmax = 0.25 / s->omega;
            long np = (long)ceil(len / hmax);
            long j;
            double h;
            if (np < 1)
                np = 1;
            h = len / (double)np;
            for (j = 0; j < np; ++j) {
                double lo = a + h * (double)j;
                double mid = lo + 0.5 * h;
                int q;
                for (q = 0; q < 4; ++q) {
                    acc += 0.5 * h * w8[q] * paper_field_x(s, mid - 0.5 * h * x8[q]);
                    acc += 0.5 * h * w8[q] * paper_field_x(s, mid + 0.5 * h * x8[q]);
                }
            }
        }
        a = b;
    }
    return -acc;
}

void orc_pulse_A(const orc_pulse *s, double t, double A[2])
{
    double amp, env;
    A[0] = 0.0;
    A[1] = 0.0;
    switch (s->kind) {
    case ORC_PULSE_ZERO:
        return;
    case ORC_PULSE_SIN2:
        amp = s->E0 / s->omega;
        env = sin(M_PI * t / s->T);
        env = env * env;
        A[0] = amp * env * sin(s->omega * t);
        A[1] = amp * env * s->eps * cos(s->omega * t);
        return;
    case ORC_PULSE_GAUSS:
        amp = s->E0 / s->omega;
        env = exp(-((t - s->t0) * (t - s->t0)) / (s->tau * s->tau));
        A[0] = amp * env * sin(s->omega * t);
        A[1] = amp * env * s->eps * cos(s->omega * t);
        return;
    case ORC_PULSE_TWO_COLOUR: {
        double w1 = s->omega, w2 = 2.0 * s->omega;
        env = sin(M_PI * t / s->T);
        env = env * env;
        A[0] = env * ((s->E0 / w1) * sin(w1 * t) + (s->E0 / w2) * sin(w2 * t + s->phase2));
        A[1] = env * s->eps *
               ((s->E0 / w1) * cos(w1 * t) + (s->E0 / w2) * cos(w2 * t + s->phase2));
        return;
    }
    case ORC_PULSE_CONST_FIELD:
        A[0] = -s->E0 * (t - 0.5 * s->T);
        return;
    case ORC_PULSE_PAPER:
        A[0] = paper_A_x(s, t);
        return;
    default:
        A[0] = NAN;
        A[1] = NAN;
    }
}

/* Time grid t_i = 0, t_f = T, dt = T/N.  a_mid[2n..2n+1] = A(t_i + (n + 1/2) dt)
 * (Sec. III, Eq. (approx_time): the step uses P at the midpoint of its own
 * interval).  a_in = A(t_i), a_out = A(t_f) (Sec. II, the asymptotic values
 * A^in, A^out).  Returns 0, or -1 on a bad argument. */
int orc_pulse_table(const orc_pulse *s, int64_t n_steps, double *a_mid, double *a_in,
                    double *a_out, double *dt_out)
{
    int64_t n;
    double dt;
    if (!s || n_steps < 0 || !(s->T > 0.0))
        return -1;
    dt = n_steps > 0 ? s->T / (double)n_steps : 0.0;
    for (n = 0; n < n_steps; ++n)
        orc_pulse_A(s, ((double)n + 0.5) * dt, a_mid + 2 * n);
    orc_pulse_A(s, 0.0, a_in);
    orc_pulse_A(s, s->T, a_out);
    *dt_out = dt;
    return 0;
}

/* Two Gauss points per step for the MAGNUS4 scheme: a_gauss[4n .. 4n+3] =
 * (A_x, A_y)(t_n + (1/2 - sqrt(3)/6) dt), (A_x, A_y)(t_n + (1/2 + sqrt(3)/6) dt). */
int orc_pulse_table_gauss(const orc_pulse *s, int64_t n_steps, double *a_gauss, double *a_in,
                          double *a_out, double *dt_out)
{
    int64_t n;
    double dt;
    const double c1 = 0.5 - sqrt(3.0) / 6.0, c2 = 0.5 + sqrt(3.0) / 6.0;
    if (!s || n_steps < 0 || !(s->T > 0.0))
        return -1;
    dt = n_steps > 0 ? s->T / (double)n_steps : 0.0;
    for (n = 0; n < n_steps; ++n) {
        orc_pulse_A(s, ((double)n + c1) * dt, a_gauss + 4 * n);
        orc_pulse_A(s, ((double)n + c2) * dt, a_gauss + 4 * n + 2);
    }
    orc_pulse_A(s, 0.0, a_in);
    orc_pulse_A(s, s->T, a_out);
    *dt_out = dt;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Free spinors, Sec. II Eq. (free_spin1..4), divided by sqrt(2E) so |u|=|v|=1 */
/* ------------------------------------------------------------------------- */

/* u: positive-energy spinor of H = valley * sigma.P.
 *   K+: u ~ [E, Px + i Py],   K-: u ~ [E, -Px - i Py]                      */
void orc_spinor_u(double Px, double Py, int valley, cplx u[2])
{
    double E = sqrt(Px * Px + Py * Py);
    double r = 1.0 / sqrt(2.0);
    /* At P = 0 the spinors are undefined; take the limit P -> (0+, 0). */
    cplx w = E > 0.0 ? (Px + I * Py) / E : 1.0;
    u[0] = r;
    u[1] = (valley > 0 ? w : -w) * r;
}

/* v: negative-energy spinor.
 *   K+: v ~ [-Px + i Py, E],  K-: v ~ [Px - i Py, E]                       */
void orc_spinor_v(double Px, double Py, int valley, cplx v[2])
{
    double E = sqrt(Px * Px + Py * Py);
    double r = 1.0 / sqrt(2.0);
    cplx w = E > 0.0 ? (-Px + I * Py) / E : -1.0; /* limit P -> (0+, 0) */
    v[0] = (valley > 0 ? w : -w) * r;
    v[1] = r;
}

/* ------------------------------------------------------------------------- */
/* One time step                                                              */
/* ------------------------------------------------------------------------- */

/* The 2x2 step operator as a matrix (row-major, m[0]=m00, m[1]=m01, ...).
 * EXACT: Sec. III closed form, U = I cos(dt E) - i (valley sigma.P/E) sin(dt E),
 *        with sigma.P = [[0, Px - i Py], [Px + i Py, 0]].  For E = 0 the
 *        limit sin(dt E)/E = dt is used.
 * STRANG_XY: U = X(a) Y(b) X(a), X(a) = cos a I - i sin a sigma_x,
 *        Y(b) = cos b I - i sin b sigma_y, a = valley dt Px/2, b = valley dt Py. */
static void step_matrix(double Px, double Py, double dt, int scheme, int valley, cplx m[4])
{
    double sg = valley > 0 ? 1.0 : -1.0;
    if (scheme == 0) {
        double E = sqrt(Px * Px + Py * Py);
        double c = cos(dt * E);
        double S = E > 0.0 ? sin(dt * E) / E : dt;
        cplx sp01 = Px - I * Py; /* (sigma.P)_{01} */
        cplx sp10 = Px + I * Py; /* (sigma.P)_{10} */
        m[0] = c;
        m[1] = -I * sg * S * sp01;
        m[2] = -I * sg * S * sp10;
        m[3] = c;
    } else {
        double a = sg * dt * Px / 2.0, b = sg * dt * Py;
        cplx X[4], Y[4], XY[4];
        X[0] = cos(a);
        X[1] = -I * sin(a);
        X[2] = -I * sin(a);
        X[3] = cos(a);
        /* sigma_y = [[0, -i], [i, 0]] so -i sin b sigma_y = [[0, -sin b], [sin b, 0]] */
        Y[0] = cos(b);
        Y[1] = -sin(b);
        Y[2] = sin(b);
        Y[3] = cos(b);
        XY[0] = X[0] * Y[0] + X[1] * Y[2];
        XY[1] = X[0] * Y[1] + X[1] * Y[3];
        XY[2] = X[2] * Y[0] + X[3] * Y[2];
        XY[3] = X[2] * Y[1] + X[3] * Y[3];
        m[0] = XY[0] * X[0] + XY[1] * X[2];
        m[1] = XY[0] * X[1] + XY[1] * X[3];
        m[2] = XY[2] * X[0] + XY[3] * X[2];
        m[3] = XY[2] * X[1] + XY[3] * X[3];
    }
}

/* MAGNUS4 step from the kinematic momenta at the two Gauss points. */
static void step_matrix_magnus4(double P1x, double P1y, double P2x, double P2y, double dt,
                                int valley, cplx m[4])
{
    double sg = valley > 0 ? 1.0 : -1.0;
    cplx A1[4], A2[4], C[4], W[4];
    double nx, ny, nz, nn, c, sn;
    int k;
    /* A_k = -i valley sigma.P_k = -i valley [[0, Px - i Py], [Px + i Py, 0]] */
    A1[0] = 0.0;
    A1[1] = -I * sg * (P1x - I * P1y);
    A1[2] = -I * sg * (P1x + I * P1y);
    A1[3] = 0.0;
    A2[0] = 0.0;
    A2[1] = -I * sg * (P2x - I * P2y);
    A2[2] = -I * sg * (P2x + I * P2y);
    A2[3] = 0.0;
    /* C = [A1, A2] = A1 A2 - A2 A1 */
    C[0] = A1[0] * A2[0] + A1[1] * A2[2] - (A2[0] * A1[0] + A2[1] * A1[2]);
    C[1] = A1[0] * A2[1] + A1[1] * A2[3] - (A2[0] * A1[1] + A2[1] * A1[3]);
    C[2] = A1[2] * A2[0] + A1[3] * A2[2] - (A2[2] * A1[0] + A2[3] * A1[2]);
    C[3] = A1[2] * A2[1] + A1[3] * A2[3] - (A2[2] * A1[1] + A2[3] * A1[3]);
    for (k = 0; k < 4; ++k)
        W[k] = 0.5 * dt * (A1[k] + A2[k]) - sqrt(3.0) * dt * dt / 12.0 * C[k];
    /* W = -i (nx sx + ny sy + nz sz): nz = i W00, nx - i ny = i W01 */
    nz = creal(I * W[0]);
    nx = creal(I * W[1]);
    ny = -cimag(I * W[1]);
    nn = sqrt(nx * nx + ny * ny + nz * nz);
    c = cos(nn);
    sn = nn > 0.0 ? sin(nn) / nn : 1.0;
    /* exp(-i n.sigma) = cos|n| I - i sin|n| (n/|n|).sigma */
    m[0] = c - I * sn * nz;
    m[1] = -I * sn * (nx - I * ny);
    m[2] = -I * sn * (nx + I * ny);
    m[3] = c + I * sn * nz;
}

void orc_step_matrix_magnus4(double P1x, double P1y, double P2x, double P2y, double dt, int valley,
                             double *out8)
{
    cplx m[4];
    int k;
    step_matrix_magnus4(P1x, P1y, P2x, P2y, dt, valley, m);
    for (k = 0; k < 4; ++k) {
        out8[2 * k] = creal(m[k]);
        out8[2 * k + 1] = cimag(m[k]);
    }
}

void orc_step_matrix(double Px, double Py, double dt, int scheme, int valley, double *out8)
{
    cplx m[4];
    int k;
    step_matrix(Px, Py, dt, scheme, valley, m);
    for (k = 0; k < 4; ++k) {
        out8[2 * k] = creal(m[k]);
        out8[2 * k + 1] = cimag(m[k]);
    }
}

/* ------------------------------------------------------------------------- */
/* Whole solve of one momentum point                                          */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double *a_mid;
    int64_t n_steps;
    double dt;
    double a_in[2], a_out[2];
    int scheme, valley;
} solve_args;

/* Evolves the point p from v(p + A_in) through all steps (Sec. III, Eq.
 * (ev_op_dt): the product of one-step operators, applied in time order) and
 * projects the result on u(p + A_out) and v(p + A_out). */
static void solve_point(const solve_args *a, double px, double py, double *cp2, double *cm2,
                        double *nrm2, double *psi_out)
{
    cplx psi[2], u[2], v[2], m[4], t0, t1, cp, cm;
    int64_t n;
    orc_spinor_v(px + a->a_in[0], py + a->a_in[1], a->valley, psi);
    for (n = 0; n < a->n_steps; ++n) {
        if (a->scheme == 2) {
            const double *g = a->a_mid + 4 * n; /* two Gauss-point samples */
            step_matrix_magnus4(px + g[0], py + g[1], px + g[2], py + g[3], a->dt, a->valley, m);
        } else {
            double Px = px + a->a_mid[2 * n];
            double Py = py + a->a_mid[2 * n + 1];
            step_matrix(Px, Py, a->dt, a->scheme, a->valley, m);
        }
        t0 = m[0] * psi[0] + m[1] * psi[1];
        t1 = m[2] * psi[0] + m[3] * psi[1];
        psi[0] = t0;
        psi[1] = t1;
    }
    {
        double Px = px + a->a_out[0], Py = py + a->a_out[1];
        if (sqrt(Px * Px + Py * Py) > 0.0) {
            orc_spinor_u(Px, Py, a->valley, u);
            orc_spinor_v(Px, Py, a->valley, v);
            cp = conj(u[0]) * psi[0] + conj(u[1]) * psi[1];
            cm = conj(v[0]) * psi[0] + conj(v[1]) * psi[1];
        } else {
            /* |P_out| = 0: the spinors are undefined; define |c+|^2 = 0. */
            cp = 0.0;
            cm = 0.0;
        }
    }
    if (cp2)
        *cp2 = creal(cp) * creal(cp) + cimag(cp) * cimag(cp);
    if (cm2)
        *cm2 = creal(cm) * creal(cm) + cimag(cm) * cimag(cm);
    if (nrm2)
        *nrm2 = creal(psi[0] * conj(psi[0]) + psi[1] * conj(psi[1]));
    if (psi_out) {
        psi_out[0] = creal(psi[0]);
        psi_out[1] = cimag(psi[0]);
        psi_out[2] = creal(psi[1]);
        psi_out[3] = cimag(psi[1]);
    }
}

static int check_common(const double *a_mid, int64_t n_steps, double dt, int scheme, int valley)
{
    if (n_steps < 0 || (n_steps > 0 && !a_mid))
        return -1;
    if (!(dt >= 0.0) || scheme < 0 || scheme > 2 || (valley != 1 && valley != -1))
        return -1;
    return 0;
}

/* Any list of momentum points: px[k], py[k].  Each output array may be NULL.
 * psi_out holds 4 doubles per point (Re a, Im a, Re b, Im b). */
int orc_solve_points(int64_t npts, const double *px, const double *py, int scheme, int valley,
                     const double *a_mid, int64_t n_steps, double dt, const double *a_in,
                     const double *a_out, double *cplus2, double *cminus2, double *norm2,
                     double *psi_out, int nthreads)
{
    solve_args a;
    int64_t k;
    if (npts < 0 || !px || !py || !a_in || !a_out)
        return -1;
    if (check_common(a_mid, n_steps, dt, scheme, valley))
        return -1;
    a.a_mid = a_mid;
    a.n_steps = n_steps;
    a.dt = dt;
    a.a_in[0] = a_in[0];
    a.a_in[1] = a_in[1];
    a.a_out[0] = a_out[0];
    a.a_out[1] = a_out[1];
    a.scheme = scheme;
    a.valley = valley;
#ifdef _OPENMP
    /* a thread count for this call only (0: all of them) */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
    for (k = 0; k < npts; ++k)
        solve_point(&a, px[k], py[k], cplus2 ? cplus2 + k : NULL, cminus2 ? cminus2 + k : NULL,
                    norm2 ? norm2 + k : NULL, psi_out ? psi_out + 4 * k : NULL);
    (void)nthreads;
    return 0;
}

/* Cell-centred grid node: the reading of a momentum interval [a, b] sampled at N points. */
double orc_grid_node(double lo, double hi, int n, int i)
{
    double h = (hi - lo) / (double)n;
    return lo + ((double)i + 0.5) * h;
}

/* Pairwise (recursive) summation, so the sum's rounding grows as log(n). */
static double pairwise_sum(const double *x, int64_t n)
{
    if (n <= 8) {
        double s = 0.0;
        int64_t i;
        for (i = 0; i < n; ++i)
            s += x[i];
        return s;
    }
    return pairwise_sum(x, n / 2) + pairwise_sum(x + n / 2, n - n / 2);
}

/* Sec. II, Eq. (pair_prod_homo) with normalised spinors and the degeneracy
 * factor 4 (two spins times two valleys): n = 4/(2 pi)^2 * hx hy * sum |c+|^2. */
double orc_density(int64_t count, const double *cplus2, double hx, double hy)
{
    return 4.0 / ((2.0 * M_PI) * (2.0 * M_PI)) * hx * hy * pairwise_sum(cplus2, count);
}

/* Whole grid, row-major [ny][nx] with x fastest.  Any output may be NULL. */
int orc_solve_grid(int32_t nx, int32_t ny, double pxmin, double pxmax, double pymin,
                   double pymax, int scheme, int valley, const double *a_mid, int64_t n_steps,
                   double dt, const double *a_in, const double *a_out, double *cplus2,
                   double *cminus2, double *norm2, double *density, int nthreads)
{
    int64_t count, k;
    double *px, *py, *cp;
    int rc;
    if (nx < 0 || ny < 0)
        return -1;
    count = (int64_t)nx * (int64_t)ny;
    px = (double *)malloc(sizeof(double) * (size_t)(count > 0 ? count : 1));
    py = (double *)malloc(sizeof(double) * (size_t)(count > 0 ? count : 1));
    cp = cplus2 ? cplus2 : (double *)malloc(sizeof(double) * (size_t)(count > 0 ? count : 1));
    if (!px || !py || !cp) {
        free(px);
        free(py);
        if (!cplus2)
            free(cp);
        return -2;
    }
    for (k = 0; k < count; ++k) {
        px[k] = orc_grid_node(pxmin, pxmax, nx, (int)(k % nx));
        py[k] = orc_grid_node(pymin, pymax, ny, (int)(k / nx));
    }
    rc = orc_solve_points(count, px, py, scheme, valley, a_mid, n_steps, dt, a_in, a_out, cp,
                          cminus2, norm2, NULL, nthreads);
    if (rc == 0 && density)
        *density = count > 0 ? orc_density(count, cp, (pxmax - pxmin) / nx, (pymax - pymin) / ny)
                             : 0.0;
    free(px);
    free(py);
    if (!cplus2)
        free(cp);
    return rc;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
