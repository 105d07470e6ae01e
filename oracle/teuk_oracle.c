/*
 * teuk_oracle.c -- plain, single-threaded FP64 reference for the Lax-Wendroff
 * time step of the (2+1)D Teukolsky equation for one azimuthal mode m.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * compared against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or constant
 * generator with the CUDA library, and it never calls the GPU.
 *
 * What it computes (Khanna & McKennon, arXiv 1001.3631, Sec. 2):
 *   Eq. (1)      Teukolsky master equation in Boyer-Lindquist coordinates.
 *   Eqs. (2)-(4) tortoise coordinate r*, azimuth phi~, ansatz Psi = e^{im phi~} r^3 Phi.
 *   Eqs. (5)-(7) Pi = d_t Phi + b d_r* Phi,  b = (r^2+a^2)/Sigma,
 *                Sigma^2 = (r^2+a^2)^2 - a^2 Delta sin^2(theta).
 *   Eqs. (8)-(12) first-order system d_t u + D d_r* u = S, u = {Phi_R,Phi_I,Pi_R,Pi_I},
 *                D = diag(b, b, -b, -b).
 *   Eq. (13)     Lax-Wendroff predictor at the half points i+1/2.
 *   Eq. (14)     Lax-Wendroff corrector at the integer points i.
 *   Sec. 2.2 (after Eq. 14): centred second-order angular differences;
 *                Phi = Pi = 0 on both radial boundaries; d_theta Phi = 0 at the
 *                poles for even |m|, Phi = 0 at the poles for odd |m| (stated for
 *                the paper's s = -2; read here as the parity of |m + s|, the same for
 *                even s and the pole behaviour of the spin-weighted harmonics,
 *                ~ theta^|m+s|, for odd s).
 *
 * The matrices M, L, A of Eq. (8) are not printed in the paper.  The source
 * vector S used here is what Eq. (1) becomes after the substitutions of
 * Eqs. (2)-(7) (the algebra is checked symbolically against Eq. (1) by the
 * test suite):
 *
 *   Phi_tt + c_t Phi_t - b^2 Phi_** - p* Phi_* - w Theta[Phi] - q Phi = tau
 *
 *   R = r^2 + a^2,  w = Delta / Sigma^2
 *   c_t = [4 i M a m r + 2 s (r Delta - M (r^2 - a^2)) + 2 i s a Delta cos(theta)] / Sigma^2
 *   p*  = w (6 R / r + 2 r) + (2 R / Sigma^2) (s (r - M) + i m a)
 *   q   = [6 Delta^2 / r^2 + 6 Delta ((s+1)(r-M) + i m a) / r + 4 i s m a (r - M)] / Sigma^2
 *   Theta[Phi] = (1/sin) d_theta(sin d_theta Phi) - [(m + s cos)^2 / sin^2 - s] Phi
 *   tau = 4 pi Delta (r^2 + a^2 cos^2) T_m / (Sigma^2 r^3)
 *
 * and with Pi = Phi_t + b Phi_*:
 *   S_Phi = Pi
 *   S_Pi  = -c_t Pi + P* Phi_* + w Theta[Phi] + q Phi + tau,   P* = c_t b + p* - b b_{,r*}
 *   b b_{,r*} = a^2 Delta sin^2 (R Delta' - 4 r Delta) / (2 Sigma^4),  Delta' = 2 (r - M).
 *
 * Readings of points the paper leaves open:
 *   grid: r* node-centred with both end points, theta cell-centred
 *         theta_j = (j + 1/2) pi / N_theta, so no node sits on a pole;
 *   S at a half point is evaluated from the averaged state, with the radial
 *         derivative taken as the one-cell difference across the half point;
 *   angular boundary conditions through one ghost row at each pole face;
 *   time step rule (Courant factor) and the synthetic source, see orc_grid();
 *   the moving-particle source (orc_run_traj) takes the circular-orbit source with
 *         the Gaussian centred on sampled particle positions.
 */
#define _USE_MATH_DEFINES
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* Problem statement: spin weight s, mode m, Kerr M and a (Eq. 1), the grid in
 * (r*, theta) (Eqs. 2-4), the Courant factor, the source orbit and the
 * extraction radius.  Mirrors, field by field, the struct the Python wrapper
 * fills; it is declared here only. */
typedef struct {
    int s, m;
    double M, a;
    double rstar_min, rstar_max;
    int n_rstar, n_theta;
    double courant;
    int dt_rule;            /* 0: dt = C dr*;  1: dt = C min(dr*, dtheta / (|m| + |s| + 2)) */
    double dt;              /* > 0 overrides the rule */
    double rstar_ext;
    double r0;              /* circular orbit radius of the synthetic source */
    double sigma_r_cells, sigma_th_cells;   /* Gaussian widths in cells */
    double sigma_r_abs, sigma_th_abs;       /* > 0 overrides the widths in cells */
} orc_params;

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------ */
/* Kerr geometry (Eq. 1: Delta = r^2 - 2 M r + a^2; Eq. 2: tortoise r*) */
/* ------------------------------------------------------------------ */

void orc_horizons(double M, double a, double* rp, double* rm) {
    double d = sqrt(M * M - a * a);
    *rp = M + d;
    *rm = M - d;
}

/* r*(r) with r = r_+ + x, the integral of Eq. (2) with the constant fixed so
 * that r* = r + 2M ln(r/2M - 1) at a = 0:
 *   r* = r + 2 M r_+/(r_+ - r_-) ln(x / 2M) - 2 M r_-/(r_+ - r_-) ln((r - r_-)/2M). */
double orc_rstar_of_x(double M, double a, double x) {
    double rp, rm;
    orc_horizons(M, a, &rp, &rm);
    double r = rp + x;
    double k = 2.0 * M / (rp - rm);
    return r + k * rp * log(x / (2.0 * M)) - k * rm * log((r - rm) / (2.0 * M));
}

/* Inverse of Eq. (2): the x = r - r_+ > 0 with r*(r_+ + x) = rstar.
 * Bisection on y = ln x (r* is strictly increasing in y); working in x keeps
 * Delta = x (x + r_+ - r_-) exact near the horizon where r - r_+ ~ 1e-27. */
double orc_x_of_rstar(double M, double a, double rstar) {
    double lo = -700.0, hi = 30.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (orc_rstar_of_x(M, a, exp(mid)) < rstar) lo = mid; else hi = mid;
    }
    return exp(0.5 * (lo + hi));
}

/* ------------------------------------------------------------------ */
/* Coefficients of S at a point (r = r_+ + x, theta)                   */
/* ------------------------------------------------------------------ */

typedef struct {
    double b, w, bbr;         /* b, Delta/Sigma^2, b b_{,r*} */
    cplx ct, pst, Pst, q;     /* c_t, p*, P* = c_t b + p* - b b_{,r*}, q */
} orc_coef;

static orc_coef coef_at(const orc_params* p, double x, double th) {
    double rp, rm;
    orc_horizons(p->M, p->a, &rp, &rm);
    const double M = p->M, a = p->a;
    const double s = (double)p->s, m = (double)p->m;
    double r = rp + x;
    double Delta = x * (x + rp - rm);
    double R = r * r + a * a;
    double sn = sin(th), cs = cos(th);
    double Sig2 = R * R - a * a * Delta * sn * sn;
    orc_coef c;
    c.b = R / sqrt(Sig2);
    c.w = Delta / Sig2;
    c.ct = (4.0 * I * M * a * m * r + 2.0 * s * (r * Delta - M * (r * r - a * a))
            + 2.0 * I * s * a * Delta * cs) / Sig2;
    c.pst = c.w * (6.0 * R / r + 2.0 * r) + (2.0 * R / Sig2) * (s * (r - M) + I * m * a);
    c.q = (6.0 * Delta * Delta / (r * r) + 6.0 * Delta * ((s + 1.0) * (r - M) + I * m * a) / r
           + 4.0 * I * s * m * a * (r - M)) / Sig2;
    c.bbr = a * a * Delta * sn * sn * (R * 2.0 * (r - M) - 4.0 * r * Delta) / (2.0 * Sig2 * Sig2);
    c.Pst = c.ct * c.b + c.pst - c.bbr;
    return c;
}

/* Pin hook: out = {b, w, bbr, Re ct, Im ct, Re p*, Im p*, Re P*, Im P*, Re q, Im q, V} */
void orc_coeffs(const orc_params* p, double x, double th, double* out) {
    orc_coef c = coef_at(p, x, th);
    double s = (double)p->s, m = (double)p->m;
    double sn = sin(th), cs = cos(th);
    out[0] = c.b; out[1] = c.w; out[2] = c.bbr;
    out[3] = creal(c.ct); out[4] = cimag(c.ct);
    out[5] = creal(c.pst); out[6] = cimag(c.pst);
    out[7] = creal(c.Pst); out[8] = cimag(c.Pst);
    out[9] = creal(c.q); out[10] = cimag(c.q);
    out[11] = (m + s * cs) * (m + s * cs) / (sn * sn) - s;
}

/* ------------------------------------------------------------------ */
/* Grid, time step and extraction point                                 */
/* ------------------------------------------------------------------ */

typedef struct {
    int nr, nth;
    double drs, dth, dt;
    double rp, rm;
    double ghost;            /* +1: even |m + s| (d_theta Phi = 0), -1: odd |m + s| (Phi = 0) */
    int i_e;                 /* extraction between i_e and i_e + 1 */
    double f_e;              /* linear weight of node i_e + 1 */
} orc_geom;

static int geom_of(const orc_params* p, orc_geom* g) {
    if (!(p->M > 0) || !(fabs(p->a) < p->M) || p->n_rstar < 4 || p->n_theta < 2 ||
        !(p->rstar_max > p->rstar_min))
        return ORC_EINVAL;
    g->nr = p->n_rstar;
    g->nth = p->n_theta;
    g->drs = (p->rstar_max - p->rstar_min) / (double)(p->n_rstar - 1);
    g->dth = M_PI / (double)p->n_theta;
    orc_horizons(p->M, p->a, &g->rp, &g->rm);
    if (p->dt > 0) {
        g->dt = p->dt;
    } else if (p->dt_rule == 0) {
        g->dt = p->courant * g->drs;
    } else if (p->dt_rule == 1) {
        double lim = g->dth / (double)(abs(p->m) + abs(p->s) + 2);
        g->dt = p->courant * (g->drs < lim ? g->drs : lim);
    } else {
        return ORC_EINVAL;
    }
    if (!(g->dt > 0)) return ORC_EINVAL;
    g->ghost = (abs(p->m + p->s) % 2 == 0) ? 1.0 : -1.0;
    double pos = (p->rstar_ext - p->rstar_min) / g->drs;
    if (!(pos >= 0.0) || !(pos <= (double)(g->nr - 1))) return ORC_EINVAL;
    int ie = (int)floor(pos);
    if (ie > g->nr - 2) ie = g->nr - 2;
    g->i_e = ie;
    g->f_e = (p->rstar_ext - (p->rstar_min + ie * g->drs)) / g->drs;
    return ORC_OK;
}

/* out = {dr*, dtheta, dt, r_+, r_-, i_e, f_e} */
int orc_grid(const orc_params* p, double* out) {
    orc_geom g;
    int st = geom_of(p, &g);
    if (st) return st;
    out[0] = g.drs; out[1] = g.dth; out[2] = g.dt; out[3] = g.rp; out[4] = g.rm;
    out[5] = (double)g.i_e; out[6] = g.f_e;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Synthetic particle source                                            */
/* ------------------------------------------------------------------ */
/*
 * The paper's source T (Eq. 1) is a Maple-generated expression that is not
 * printed (Sec. 2.1, Sec. 3).  It is replaced by a point particle on a
 * circular equatorial orbit at r0, smeared by a 2D Gaussian in (r*, theta):
 *   T_m(t, r*, theta) = A_n exp(-i m (Omega t + phi0)) G(r* - r*(r0), theta - pi/2)
 *   G = exp(-(dr^2/sig_r^2 + dth^2/sig_th^2)/2) / (2 pi sig_r sig_th), zero beyond 8 sigma
 *   Omega = M^(1/2) / (r0^(3/2) + a M^(1/2))            (prograde circular Kerr orbit)
 *   phi0  = a/(r_+ - r_-) ln((r0 - r_+)/(r0 - r_-))      (the phi~ shift of Eq. 3 at r0)
 * and enters S_Pi as tau = 4 pi Delta (r^2 + a^2 cos^2) T_m / (Sigma^2 r^3).
 * So tau(t_n) = A_n exp(-i (omega t + phase0)) P(r*, theta) with omega = m Omega,
 * phase0 = m phi0 and a static profile P.
 */

/* out = {Omega, phi0, r*0, r_ext, dOmega/dr0, dphi0/dr0, dr*0/dr0, sigma_r, sigma_th, x0} */
int orc_orbit(const orc_params* p, double* out) {
    orc_geom g;
    int st = geom_of(p, &g);
    if (st) return st;
    double M = p->M, a = p->a, r0 = p->r0;
    if (!(r0 > g.rp)) return ORC_EINVAL;
    double sq = sqrt(M);
    double den = pow(r0, 1.5) + a * sq;
    double Omega = sq / den;
    double phi0 = a / (g.rp - g.rm) * log((r0 - g.rp) / (r0 - g.rm));
    double x0 = r0 - g.rp;
    double rs0 = orc_rstar_of_x(M, a, x0);
    double xe = orc_x_of_rstar(M, a, p->rstar_ext);
    double Delta0 = r0 * r0 - 2.0 * M * r0 + a * a;
    out[0] = Omega;
    out[1] = phi0;
    out[2] = rs0;
    out[3] = g.rp + xe;
    out[4] = -sq * 1.5 * sqrt(r0) / (den * den);
    out[5] = a / Delta0;
    out[6] = (r0 * r0 + a * a) / Delta0;
    out[7] = p->sigma_r_abs > 0 ? p->sigma_r_abs : p->sigma_r_cells * g.drs;
    out[8] = p->sigma_th_abs > 0 ? p->sigma_th_abs : p->sigma_th_cells * g.dth;
    out[9] = x0;
    return ORC_OK;
}

/* P and dP/dr0 (both without the time phase) at one point. */
static void profile_at(const orc_params* p, const double* orb, double x, double rs, double th,
                       cplx* P, cplx* dP) {
    double sig_r = orb[7], sig_t = orb[8];
    double dr = rs - orb[2], dt = th - 0.5 * M_PI;
    if (fabs(dr) > 8.0 * sig_r || fabs(dt) > 8.0 * sig_t) { *P = 0; *dP = 0; return; }
    double G = exp(-0.5 * (dr * dr / (sig_r * sig_r) + dt * dt / (sig_t * sig_t)))
               / (2.0 * M_PI * sig_r * sig_t);
    double rp, rm;
    orc_horizons(p->M, p->a, &rp, &rm);
    double a = p->a;
    double r = rp + x;
    double Delta = x * (x + rp - rm);
    double R = r * r + a * a;
    double sn = sin(th), cs = cos(th);
    double Sig2 = R * R - a * a * Delta * sn * sn;
    double pref = 4.0 * M_PI * (r * r + a * a * cs * cs) * Delta / (Sig2 * r * r * r);
    *P = pref * G;
    /* d/dr0 G(r* - r*0(r0)) = G (r* - r*0)/sig_r^2 * dr*0/dr0 */
    *dP = pref * G * dr / (sig_r * sig_r) * orb[6];
}

/* Profiles on the grid: P_int, dP_int [nth][nr] at (r*_i, theta_j);
 * P_half, dP_half [nth][nr-1] at (r*_{i+1/2}, theta_j).  Complex arrays as
 * interleaved (re, im) doubles. */
int orc_orbit_profile(const orc_params* p, double* P_int, double* P_half, double* dP_int,
                      double* dP_half) {
    orc_geom g;
    int st = geom_of(p, &g);
    if (st) return st;
    double orb[10];
    st = orc_orbit(p, orb);
    if (st) return st;
    cplx *Pi_ = (cplx*)P_int, *Ph = (cplx*)P_half, *dPi = (cplx*)dP_int, *dPh = (cplx*)dP_half;
    /* r at each column, once (the inversion does not depend on theta) */
    double* xi = malloc(sizeof(double) * g.nr);
    double* xh = malloc(sizeof(double) * g.nr);
    if (!xi || !xh) { free(xi); free(xh); return ORC_ENOMEM; }
    for (int i = 0; i < g.nr; ++i) xi[i] = orc_x_of_rstar(p->M, p->a, p->rstar_min + i * g.drs);
    for (int i = 0; i < g.nr - 1; ++i)
        xh[i] = orc_x_of_rstar(p->M, p->a, p->rstar_min + (i + 0.5) * g.drs);
    for (int j = 0; j < g.nth; ++j) {
        double th = (j + 0.5) * g.dth;
        for (int i = 0; i < g.nr; ++i) {
            double rs = p->rstar_min + i * g.drs;
            profile_at(p, orb, xi[i], rs, th, &Pi_[(size_t)j * g.nr + i], &dPi[(size_t)j * g.nr + i]);
        }
        for (int i = 0; i < g.nr - 1; ++i) {
            double rs = p->rstar_min + (i + 0.5) * g.drs;
            profile_at(p, orb, xh[i], rs, th, &Ph[(size_t)j * (g.nr - 1) + i],
                       &dPh[(size_t)j * (g.nr - 1) + i]);
        }
    }
    free(xi);
    free(xh);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Lax-Wendroff step (Eqs. 13-14)                                       */
/* ------------------------------------------------------------------ */

typedef struct {
    orc_params p;
    orc_geom g;
    orc_coef* ci;     /* [nth][nr]    coefficients at (r*_i, theta_j) */
    orc_coef* ch;     /* [nth][nr-1]  coefficients at (r*_{i+1/2}, theta_j) */
    double* cot;      /* [nth] cot(theta_j) */
    double* V;        /* [nth] (m + s cos)^2/sin^2 - s */
} orc_ctx;

static void ctx_free(orc_ctx* c) {
    free(c->ci); free(c->ch); free(c->cot); free(c->V);
}

static int ctx_init(orc_ctx* c, const orc_params* p) {
    memset(c, 0, sizeof(*c));
    c->p = *p;
    int st = geom_of(p, &c->g);
    if (st) return st;
    int nr = c->g.nr, nth = c->g.nth;
    c->ci = malloc(sizeof(orc_coef) * (size_t)nr * nth);
    c->ch = malloc(sizeof(orc_coef) * (size_t)(nr - 1) * nth);
    c->cot = malloc(sizeof(double) * nth);
    c->V = malloc(sizeof(double) * nth);
    if (!c->ci || !c->ch || !c->cot || !c->V) { ctx_free(c); return ORC_ENOMEM; }
    double* xi = malloc(sizeof(double) * nr);
    double* xh = malloc(sizeof(double) * (nr - 1));
    if (!xi || !xh) { free(xi); free(xh); ctx_free(c); return ORC_ENOMEM; }
    for (int i = 0; i < nr; ++i) xi[i] = orc_x_of_rstar(p->M, p->a, p->rstar_min + i * c->g.drs);
    for (int i = 0; i < nr - 1; ++i)
        xh[i] = orc_x_of_rstar(p->M, p->a, p->rstar_min + (i + 0.5) * c->g.drs);
    for (int j = 0; j < nth; ++j) {
        double th = (j + 0.5) * c->g.dth;
        double s = (double)p->s, m = (double)p->m;
        c->cot[j] = cos(th) / sin(th);
        c->V[j] = (m + s * cos(th)) * (m + s * cos(th)) / (sin(th) * sin(th)) - s;
        for (int i = 0; i < nr; ++i) c->ci[(size_t)j * nr + i] = coef_at(p, xi[i], th);
        for (int i = 0; i < nr - 1; ++i) c->ch[(size_t)j * (nr - 1) + i] = coef_at(p, xh[i], th);
    }
    free(xi); free(xh);
    return ORC_OK;
}

/* Row jj of a field F[nth][ncol] with the angular boundary condition applied
 * through ghost rows: row -1 mirrors row 0 and row nth mirrors row nth-1,
 * with sign +1 for even |m + s| (d_theta Phi = 0 at the pole face) and -1 for
 * odd |m + s| (Phi = 0 at the pole face). */
static cplx row_val(const orc_ctx* c, const cplx* F, int ncol, int jj, int i) {
    int nth = c->g.nth;
    if (jj < 0) return c->g.ghost * F[(size_t)0 * ncol + i];
    if (jj >= nth) return c->g.ghost * F[(size_t)(nth - 1) * ncol + i];
    return F[(size_t)jj * ncol + i];
}

/* Centred second-order Theta[F] at row j (Sec. 2.2): F_thth + cot F_th - V F. */
static cplx theta_op(const orc_ctx* c, int j, cplx Fm, cplx F0, cplx Fp) {
    double h = c->g.dth;
    return (Fp - 2.0 * F0 + Fm) / (h * h) + c->cot[j] * (Fp - Fm) / (2.0 * h) - c->V[j] * F0;
}

/* Pin hook: out[j] = Theta_h[F]_j for one column F[nth] (interleaved complex),
 * with the ghost rows of the angular boundary condition. */
int orc_theta_apply(const orc_params* p, const double* F, double* out) {
    orc_ctx c;
    int st = ctx_init(&c, p);
    if (st) return st;
    const cplx* f = (const cplx*)F;
    cplx* o = (cplx*)out;
    for (int j = 0; j < c.g.nth; ++j)
        o[j] = theta_op(&c, j, row_val(&c, f, 1, j - 1, 0), f[j], row_val(&c, f, 1, j + 1, 0));
    ctx_free(&c);
    return ORC_OK;
}

/* One full step u^n -> u^{n+1} (both as complex Phi, Pi [nth][nr]).
 * tau_p = src_p * P_half is the source at (t_n, r*_{i+1/2}); tau_c = src_c * P_int
 * at (t_n + dt/2, r*_i).  hPhi, hPi [nth][nr-1] receive u^{n+1/2}_{i+1/2}. */
static void lw_step(const orc_ctx* c, const cplx* Phi, const cplx* Pi, cplx src_p, cplx src_c,
                    const cplx* P_int, const cplx* P_half, cplx* hPhi, cplx* hPi,
                    cplx* Phi1, cplx* Pi1) {
    const int nr = c->g.nr, nth = c->g.nth, nh = nr - 1;
    const double drs = c->g.drs, dt = c->g.dt;

    /* Eq. (13): u^{n+1/2}_{i+1/2} = (u_{i+1} + u_i)/2 - dt/2 [D (u_{i+1} - u_i)/dr* - S^n_{i+1/2}] */
    for (int j = 0; j < nth; ++j) {
        for (int i = 0; i < nh; ++i) {
            const orc_coef* k = &c->ch[(size_t)j * nh + i];
            cplx Phib = 0.5 * (Phi[(size_t)j * nr + i + 1] + Phi[(size_t)j * nr + i]);
            cplx Pib = 0.5 * (Pi[(size_t)j * nr + i + 1] + Pi[(size_t)j * nr + i]);
            cplx dPhi = (Phi[(size_t)j * nr + i + 1] - Phi[(size_t)j * nr + i]) / drs;
            cplx dPi = (Pi[(size_t)j * nr + i + 1] - Pi[(size_t)j * nr + i]) / drs;
            cplx Phib_m = 0.5 * (row_val(c, Phi, nr, j - 1, i + 1) + row_val(c, Phi, nr, j - 1, i));
            cplx Phib_p = 0.5 * (row_val(c, Phi, nr, j + 1, i + 1) + row_val(c, Phi, nr, j + 1, i));
            cplx tau = src_p * P_half[(size_t)j * nh + i];
            cplx S_Phi = Pib;
            cplx S_Pi = -k->ct * Pib + k->Pst * dPhi + k->w * theta_op(c, j, Phib_m, Phib, Phib_p)
                        + k->q * Phib + tau;
            hPhi[(size_t)j * nh + i] = Phib - 0.5 * dt * (k->b * dPhi - S_Phi);
            hPi[(size_t)j * nh + i] = Pib - 0.5 * dt * (-k->b * dPi - S_Pi);
        }
    }
    /* Eq. (14): u^{n+1}_i = u^n_i - dt [D (u_{i+1/2} - u_{i-1/2})/dr* - S^{n+1/2}_i] */
    for (int j = 0; j < nth; ++j) {
        for (int i = 1; i < nr - 1; ++i) {
            const orc_coef* k = &c->ci[(size_t)j * nr + i];
            /* half point i+1/2 is stored at index i, i-1/2 at index i-1 */
            cplx Phib = 0.5 * (hPhi[(size_t)j * nh + i] + hPhi[(size_t)j * nh + i - 1]);
            cplx Pib = 0.5 * (hPi[(size_t)j * nh + i] + hPi[(size_t)j * nh + i - 1]);
            cplx dPhi = (hPhi[(size_t)j * nh + i] - hPhi[(size_t)j * nh + i - 1]) / drs;
            cplx dPi = (hPi[(size_t)j * nh + i] - hPi[(size_t)j * nh + i - 1]) / drs;
            cplx Phib_m = 0.5 * (row_val(c, hPhi, nh, j - 1, i) + row_val(c, hPhi, nh, j - 1, i - 1));
            cplx Phib_p = 0.5 * (row_val(c, hPhi, nh, j + 1, i) + row_val(c, hPhi, nh, j + 1, i - 1));
            cplx tau = src_c * P_int[(size_t)j * nr + i];
            cplx S_Phi = Pib;
            cplx S_Pi = -k->ct * Pib + k->Pst * dPhi + k->w * theta_op(c, j, Phib_m, Phib, Phib_p)
                        + k->q * Phib + tau;
            Phi1[(size_t)j * nr + i] = Phi[(size_t)j * nr + i] - dt * (k->b * dPhi - S_Phi);
            Pi1[(size_t)j * nr + i] = Pi[(size_t)j * nr + i] - dt * (-k->b * dPi - S_Pi);
        }
        /* radial boundary condition: Phi = Pi = 0 at the inner and outer r* boundary */
        Phi1[(size_t)j * nr + 0] = 0; Pi1[(size_t)j * nr + 0] = 0;
        Phi1[(size_t)j * nr + nr - 1] = 0; Pi1[(size_t)j * nr + nr - 1] = 0;
    }
}

/* Waveform record: Phi at r*_ext, linear between the bracketing nodes. */
static void extract(const orc_ctx* c, const cplx* Phi, double* rec /* [nth][2] */) {
    for (int j = 0; j < c->g.nth; ++j) {
        cplx v = (1.0 - c->g.f_e) * Phi[(size_t)j * c->g.nr + c->g.i_e]
                 + c->g.f_e * Phi[(size_t)j * c->g.nr + c->g.i_e + 1];
        rec[2 * j] = creal(v);
        rec[2 * j + 1] = cimag(v);
    }
}

static double amp_of(const double* amps, int64_t n_amps, int64_t n) {
    return (amps && n < n_amps) ? amps[n] : 1.0;
}

/* Source factors of step n: A_n exp(-i (omega t + phase0)) at t_n and t_n + dt/2. */
static void src_factors(const orc_ctx* c, double omega, double phase0, const double* amps,
                        int64_t n_amps, int64_t n, cplx* sp, cplx* sc) {
    double A = amp_of(amps, n_amps, n);
    double t = (double)n * c->g.dt;
    *sp = A * cexp(-I * (omega * t + phase0));
    *sc = A * cexp(-I * (omega * (t + 0.5 * c->g.dt) + phase0));
}

static void u_to_cplx(const orc_ctx* c, const double* u, cplx* Phi, cplx* Pi) {
    size_t np = (size_t)c->g.nr * c->g.nth;
    for (size_t k = 0; k < np; ++k) {
        Phi[k] = u[k] + I * u[np + k];
        Pi[k] = u[2 * np + k] + I * u[3 * np + k];
    }
}

static void cplx_to_u(const orc_ctx* c, const cplx* Phi, const cplx* Pi, double* u) {
    size_t np = (size_t)c->g.nr * c->g.nth;
    for (size_t k = 0; k < np; ++k) {
        u[k] = creal(Phi[k]); u[np + k] = cimag(Phi[k]);
        u[2 * np + k] = creal(Pi[k]); u[3 * np + k] = cimag(Pi[k]);
    }
}

/*
 * Evolve nsteps full steps starting at global step index step0 (t = step0 dt).
 * u: [4][nth][nr] = {Phi_R, Phi_I, Pi_R, Pi_I}, in/out.
 * Source: tau = A_n exp(-i (omega t + phase0)) P with P given at integer and
 * half nodes (interleaved complex).  P_int == NULL means no source.
 * wave (optional): [(nsteps+1)][nth][2], record k is the extraction of
 * u^{step0 + k}.
 */
int orc_run(const orc_params* p, double omega, double phase0, const double* P_int,
            const double* P_half, const double* amps, int64_t n_amps, int64_t step0,
            int64_t nsteps, double* u, double* wave) {
    orc_ctx c;
    int st = ctx_init(&c, p);
    if (st) return st;
    const int nr = c.g.nr, nth = c.g.nth;
    size_t np = (size_t)nr * nth, nhp = (size_t)(nr - 1) * nth;
    cplx* Phi = malloc(sizeof(cplx) * np);
    cplx* Pi = malloc(sizeof(cplx) * np);
    cplx* Phi1 = malloc(sizeof(cplx) * np);
    cplx* Pi1 = malloc(sizeof(cplx) * np);
    cplx* hPhi = malloc(sizeof(cplx) * nhp);
    cplx* hPi = malloc(sizeof(cplx) * nhp);
    cplx* zi = calloc(np, sizeof(cplx));
    cplx* zh = calloc(nhp, sizeof(cplx));
    if (!Phi || !Pi || !Phi1 || !Pi1 || !hPhi || !hPi || !zi || !zh) {
        st = ORC_ENOMEM;
        goto done;
    }
    const cplx* Pi_src = P_int ? (const cplx*)P_int : zi;
    const cplx* Ph_src = P_half ? (const cplx*)P_half : zh;
    u_to_cplx(&c, u, Phi, Pi);
    if (wave) extract(&c, Phi, wave);
    for (int64_t k = 0; k < nsteps; ++k) {
        cplx sp, sc;
        src_factors(&c, omega, phase0, amps, n_amps, step0 + k, &sp, &sc);
        lw_step(&c, Phi, Pi, sp, sc, Pi_src, Ph_src, hPhi, hPi, Phi1, Pi1);
        cplx* t;
        t = Phi; Phi = Phi1; Phi1 = t;
        t = Pi; Pi = Pi1; Pi1 = t;
        if (wave) extract(&c, Phi, wave + (size_t)(k + 1) * 2 * nth);
    }
    cplx_to_u(&c, Phi, Pi, u);
done:
    free(Phi); free(Pi); free(Phi1); free(Pi1); free(hPhi); free(hPi); free(zi); free(zh);
    ctx_free(&c);
    return st;
}

/* ------------------------------------------------------------------ */
/* Moving particle: a sampled trajectory                                */
/* ------------------------------------------------------------------ */
/*
 * A particle on a general (eccentric or inclined) orbit, known through samples of
 * its position and amplitude taken every half step:
 *   traj[k] = {r_p, theta_p, phi_p, A} at t = k dt/2,  k = 0 .. n_samples - 1.
 * The source at sample k is the circular-orbit source above with the Gaussian
 * centred on the particle and the phase of its azimuth:
 *   tau_k(r*, theta) = A_k exp(-i m phi_p,k) pref(r, theta) G(r* - r*(r_p,k), theta - theta_p,k)
 *   pref = 4 pi Delta (r^2 + a^2 cos^2) / (Sigma^2 r^3),  G as above, zero beyond 8 sigma.
 * Step n takes sample 2n in Eq. (13) (time t_n, half nodes) and sample 2n + 1 in
 * Eq. (14) (time t_n + dt/2, integer nodes); a sub-step with no sample has no source.
 * With r_p = r0, theta_p = pi/2, phi_p = Omega t + phi0 and A_{2n} = A_{2n+1} = A_n it
 * is the circular-orbit source.
 */

/* tau of one sample at every node of one kind (integer nodes: half = 0, nodes
 * r*_min + i dr*; half nodes: half = 1, nodes r*_min + (i + 1/2) dr*), into
 * out[nth][n_nodes]; xs[i] = r - r_+ at those nodes. */
static int moving_tau(const orc_params* p, const orc_geom* g, const double* xs, int n_nodes,
                      int half, const double* smp, double sig_r, double sig_t, cplx* out) {
    double r_p = smp[0], th_p = smp[1], phi_p = smp[2], A = smp[3];
    if (!(r_p > g->rp) || !isfinite(th_p) || !isfinite(phi_p) || !isfinite(A)) return ORC_EINVAL;
    double rs_p = orc_rstar_of_x(p->M, p->a, r_p - g->rp);
    cplx amp = A * cexp(-I * ((double)p->m * phi_p));
    const double a = p->a;
    for (int j = 0; j < g->nth; ++j) {
        double th = (j + 0.5) * g->dth;
        double dth_ = th - th_p;
        for (int i = 0; i < n_nodes; ++i) {
            double rs = p->rstar_min + (half ? (i + 0.5) : (double)i) * g->drs;
            double dr = rs - rs_p;
            cplx* o = &out[(size_t)j * n_nodes + i];
            if (fabs(dr) > 8.0 * sig_r || fabs(dth_) > 8.0 * sig_t) { *o = 0; continue; }
            double G = exp(-0.5 * (dr * dr / (sig_r * sig_r) + dth_ * dth_ / (sig_t * sig_t)))
                       / (2.0 * M_PI * sig_r * sig_t);
            double x = xs[i];
            double r = g->rp + x;
            double Delta = x * (x + g->rp - g->rm);
            double R = r * r + a * a;
            double sn = sin(th), cs = cos(th);
            double Sig2 = R * R - a * a * Delta * sn * sn;
            double pref = 4.0 * M_PI * (r * r + a * a * cs * cs) * Delta / (Sig2 * r * r * r);
            *o = amp * (pref * G);
        }
    }
    return ORC_OK;
}

/*
 * Evolve nsteps full steps from global step step0 with the sampled-trajectory source
 * (arrays as in orc_run; traj [n_samples][4] as above; widths from the sigma fields
 * of p, r0 unused).
 */
int orc_run_traj(const orc_params* p, const double* traj, int64_t n_samples, int64_t step0,
                 int64_t nsteps, double* u, double* wave) {
    orc_ctx c;
    int st = ctx_init(&c, p);
    if (st) return st;
    const int nr = c.g.nr, nth = c.g.nth;
    const double sig_r = p->sigma_r_abs > 0 ? p->sigma_r_abs : p->sigma_r_cells * c.g.drs;
    const double sig_t = p->sigma_th_abs > 0 ? p->sigma_th_abs : p->sigma_th_cells * c.g.dth;
    size_t np = (size_t)nr * nth, nhp = (size_t)(nr - 1) * nth;
    cplx* Phi = malloc(sizeof(cplx) * np);
    cplx* Pi = malloc(sizeof(cplx) * np);
    cplx* Phi1 = malloc(sizeof(cplx) * np);
    cplx* Pi1 = malloc(sizeof(cplx) * np);
    cplx* hPhi = malloc(sizeof(cplx) * nhp);
    cplx* hPi = malloc(sizeof(cplx) * nhp);
    cplx* ti = malloc(sizeof(cplx) * np);
    cplx* th_ = malloc(sizeof(cplx) * nhp);
    double* xi = malloc(sizeof(double) * nr);
    double* xh = malloc(sizeof(double) * nr);
    if (!Phi || !Pi || !Phi1 || !Pi1 || !hPhi || !hPi || !ti || !th_ || !xi || !xh) {
        st = ORC_ENOMEM;
        goto done;
    }
    if (!(sig_r > 0) || !(sig_t > 0) || n_samples < 0 || (n_samples > 0 && !traj)) {
        st = ORC_EINVAL;
        goto done;
    }
    for (int i = 0; i < nr; ++i) xi[i] = orc_x_of_rstar(p->M, p->a, p->rstar_min + i * c.g.drs);
    for (int i = 0; i < nr - 1; ++i)
        xh[i] = orc_x_of_rstar(p->M, p->a, p->rstar_min + (i + 0.5) * c.g.drs);
    u_to_cplx(&c, u, Phi, Pi);
    if (wave) extract(&c, Phi, wave);
    for (int64_t k = 0; k < nsteps; ++k) {
        int64_t n = step0 + k;
        if (2 * n < n_samples) {
            st = moving_tau(p, &c.g, xh, nr - 1, 1, traj + 4 * (2 * n), sig_r, sig_t, th_);
            if (st) goto done;
        } else {
            memset(th_, 0, sizeof(cplx) * nhp);
        }
        if (2 * n + 1 < n_samples) {
            st = moving_tau(p, &c.g, xi, nr, 0, traj + 4 * (2 * n + 1), sig_r, sig_t, ti);
            if (st) goto done;
        } else {
            memset(ti, 0, sizeof(cplx) * np);
        }
        lw_step(&c, Phi, Pi, 1.0, 1.0, ti, th_, hPhi, hPi, Phi1, Pi1);
        cplx* t;
        t = Phi; Phi = Phi1; Phi1 = t;
        t = Pi; Pi = Pi1; Pi1 = t;
        if (wave) extract(&c, Phi, wave + (size_t)(k + 1) * 2 * nth);
    }
    cplx_to_u(&c, Phi, Pi, u);
done:
    free(Phi); free(Pi); free(Phi1); free(Pi1); free(hPhi); free(hPi); free(ti); free(th_);
    free(xi); free(xh);
    ctx_free(&c);
    return st;
}

/* ------------------------------------------------------------------ */
/* Adjoint (transpose) of one step                                      */
/* ------------------------------------------------------------------ */
/*
 * The step is affine and complex-linear in u:  u^{n+1} = K u^n + A_n s_n.
 * With the real inner product <x, y> = sum Re(conj(x) y) over all nodes and
 * components, the transpose of y += c x is  lx += conj(c) ly.  The adjoint
 * step below visits the forward step's operations and applies that rule to
 * each one (a scatter), in reverse order: first the corrector, then the
 * predictor.  It also returns the two inner products that give the gradient
 * with respect to the step's source:
 *   gp = <mu, dt/2 (0, tau_p)>   (predictor source, with mu = C^T lambda)
 *   gc = <lambda', dt (0, tau_c)> (corrector source)
 */
static void lw_step_adj(const orc_ctx* c, const cplx* lPhi1, const cplx* lPi1, cplx* lPhi,
                        cplx* lPi, cplx* mPhi, cplx* mPi, cplx* lPhi1_int, cplx* lPi1_int) {
    const int nr = c->g.nr, nth = c->g.nth, nh = nr - 1;
    const double drs = c->g.drs, dt = c->g.dt;
    const double gs = c->g.ghost;
    size_t np = (size_t)nr * nth, nhp = (size_t)nh * nth;
    /* radial boundary rows are overwritten with zero by the forward step */
    for (size_t k = 0; k < np; ++k) { lPhi1_int[k] = lPhi1[k]; lPi1_int[k] = lPi1[k]; }
    for (int j = 0; j < nth; ++j) {
        lPhi1_int[(size_t)j * nr] = 0; lPi1_int[(size_t)j * nr] = 0;
        lPhi1_int[(size_t)j * nr + nr - 1] = 0; lPi1_int[(size_t)j * nr + nr - 1] = 0;
    }
    for (size_t k = 0; k < np; ++k) { lPhi[k] = 0; lPi[k] = 0; }
    for (size_t k = 0; k < nhp; ++k) { mPhi[k] = 0; mPi[k] = 0; }

    /* transpose of Eq. (14) */
    for (int j = 0; j < nth; ++j) {
        for (int i = 1; i < nr - 1; ++i) {
            const orc_coef* k = &c->ci[(size_t)j * nr + i];
            cplx LF = lPhi1_int[(size_t)j * nr + i];
            cplx LP = lPi1_int[(size_t)j * nr + i];
            /* Phi1 = Phi - dt (b dPhi - Pib);  Pi1 = Pi - dt (-b dPi - S_Pi) */
            lPhi[(size_t)j * nr + i] += LF;
            lPi[(size_t)j * nr + i] += LP;
            /* dPhi = (hPhi_i - hPhi_{i-1})/drs, Pib = (hPi_i + hPi_{i-1})/2 in half indices */
            cplx gPhib = 0, gPib = 0, gdPhi = 0, gdPi = 0, gPhib_m = 0, gPhib_p = 0;
            gdPhi += -dt * k->b * LF;
            gPib += dt * LF;
            gdPi += dt * k->b * LP;
            /* dt * S_Pi, S_Pi = -ct Pib + Pst dPhi + w Theta(Phib_m, Phib, Phib_p) + q Phib */
            gPib += dt * conj(-k->ct) * LP;
            gdPhi += dt * conj(k->Pst) * LP;
            double h2 = c->g.dth * c->g.dth, h1 = 2.0 * c->g.dth;
            gPhib_p += dt * k->w * (1.0 / h2 + c->cot[j] / h1) * LP;
            gPhib_m += dt * k->w * (1.0 / h2 - c->cot[j] / h1) * LP;
            gPhib += dt * k->w * (-2.0 / h2 - c->V[j]) * LP;
            gPhib += dt * conj(k->q) * LP;
            /* scatter onto the half-state */
            mPhi[(size_t)j * nh + i] += 0.5 * gPhib + gdPhi / drs;
            mPhi[(size_t)j * nh + i - 1] += 0.5 * gPhib - gdPhi / drs;
            mPi[(size_t)j * nh + i] += 0.5 * gPib + gdPi / drs;
            mPi[(size_t)j * nh + i - 1] += 0.5 * gPib - gdPi / drs;
            /* rows j-1, j+1 (with ghost folding onto rows 0 / nth-1) */
            int jm = j - 1, jp = j + 1;
            double sm = 1.0, sp = 1.0;
            if (jm < 0) { jm = 0; sm = gs; }
            if (jp >= nth) { jp = nth - 1; sp = gs; }
            mPhi[(size_t)jm * nh + i] += 0.5 * sm * gPhib_m;
            mPhi[(size_t)jm * nh + i - 1] += 0.5 * sm * gPhib_m;
            mPhi[(size_t)jp * nh + i] += 0.5 * sp * gPhib_p;
            mPhi[(size_t)jp * nh + i - 1] += 0.5 * sp * gPhib_p;
        }
    }
    /* transpose of Eq. (13) */
    for (int j = 0; j < nth; ++j) {
        for (int i = 0; i < nh; ++i) {
            const orc_coef* k = &c->ch[(size_t)j * nh + i];
            cplx MF = mPhi[(size_t)j * nh + i];
            cplx MP = mPi[(size_t)j * nh + i];
            /* hPhi = Phib - dt/2 (b dPhi - Pib); hPi = Pib - dt/2 (-b dPi - S_Pi) */
            cplx gPhib = 0, gPib = 0, gdPhi = 0, gdPi = 0, gPhib_m = 0, gPhib_p = 0;
            gPhib += MF;
            gdPhi += -0.5 * dt * k->b * MF;
            gPib += 0.5 * dt * MF;
            gPib += MP;
            gdPi += 0.5 * dt * k->b * MP;
            gPib += 0.5 * dt * conj(-k->ct) * MP;
            gdPhi += 0.5 * dt * conj(k->Pst) * MP;
            double h2 = c->g.dth * c->g.dth, h1 = 2.0 * c->g.dth;
            gPhib_p += 0.5 * dt * k->w * (1.0 / h2 + c->cot[j] / h1) * MP;
            gPhib_m += 0.5 * dt * k->w * (1.0 / h2 - c->cot[j] / h1) * MP;
            gPhib += 0.5 * dt * k->w * (-2.0 / h2 - c->V[j]) * MP;
            gPhib += 0.5 * dt * conj(k->q) * MP;
            lPhi[(size_t)j * nr + i + 1] += 0.5 * gPhib + gdPhi / drs;
            lPhi[(size_t)j * nr + i] += 0.5 * gPhib - gdPhi / drs;
            lPi[(size_t)j * nr + i + 1] += 0.5 * gPib + gdPi / drs;
            lPi[(size_t)j * nr + i] += 0.5 * gPib - gdPi / drs;
            int jm = j - 1, jp = j + 1;
            double sm = 1.0, sp = 1.0;
            if (jm < 0) { jm = 0; sm = gs; }
            if (jp >= nth) { jp = nth - 1; sp = gs; }
            lPhi[(size_t)jm * nr + i + 1] += 0.5 * sm * gPhib_m;
            lPhi[(size_t)jm * nr + i] += 0.5 * sm * gPhib_m;
            lPhi[(size_t)jp * nr + i + 1] += 0.5 * sp * gPhib_p;
            lPhi[(size_t)jp * nr + i] += 0.5 * sp * gPhib_p;
        }
    }
}

/* Pin hooks: y = K x (one step, no source) and x = K^T y, on [4][nth][nr] arrays. */
int orc_apply_K(const orc_params* p, const double* x, double* y) {
    return orc_run(p, 0.0, 0.0, NULL, NULL, NULL, 0, 0, 1, memcpy(y, x, sizeof(double) * 4 *
                   (size_t)p->n_rstar * p->n_theta), NULL);
}

int orc_apply_KT(const orc_params* p, const double* y, double* x) {
    orc_ctx c;
    int st = ctx_init(&c, p);
    if (st) return st;
    size_t np = (size_t)c.g.nr * c.g.nth, nhp = (size_t)(c.g.nr - 1) * c.g.nth;
    cplx* buf = malloc(sizeof(cplx) * (6 * np + 2 * nhp));
    if (!buf) { ctx_free(&c); return ORC_ENOMEM; }
    cplx *lF1 = buf, *lP1 = buf + np, *lF = buf + 2 * np, *lP = buf + 3 * np;
    cplx *iF = buf + 4 * np, *iP = buf + 5 * np, *mF = buf + 6 * np, *mP = mF + nhp;
    u_to_cplx(&c, y, lF1, lP1);
    lw_step_adj(&c, lF1, lP1, lF, lP, mF, mP, iF, iP);
    cplx_to_u(&c, lF, lP, x);
    free(buf);
    ctx_free(&c);
    return ORC_OK;
}

/*
 * Reverse sweep over steps step0 .. step0+nsteps-1 for a loss L(W) of the
 * waveform records W_k = E u^{step0+k}, k = 1..nsteps.
 *   gwave   [nsteps][nth][2]: dL/dW_k (real and imaginary parts), k = 1..nsteps
 *   P, dP   profiles and their r0-derivatives at integer and half nodes
 *   domega, dphase0: d omega/d r0 and d phase0/d r0
 * Out: grad_amps[k] = dL/dA_{step0+k}, *grad_r0 = dL/dr0 and, if lam0 != NULL,
 *      lam0 [4][nth][nr] = dL/du^{step0}.
 * Recurrence: lambda^{n} = K^T lambda^{n+1} + E^T dL/dW_n, starting from
 * lambda^{N} = E^T dL/dW_N.  The problem is linear, so no forward state is
 * needed.
 */
int orc_adjoint(const orc_params* p, double omega, double phase0, const double* P_int,
                const double* P_half, const double* dP_int, const double* dP_half,
                double domega, double dphase0, const double* amps, int64_t n_amps,
                int64_t step0, int64_t nsteps, const double* gwave, double* grad_amps,
                double* grad_r0, double* lam0) {
    orc_ctx c;
    int st = ctx_init(&c, p);
    if (st) return st;
    const int nr = c.g.nr, nth = c.g.nth, nh = nr - 1;
    size_t np = (size_t)nr * nth, nhp = (size_t)nh * nth;
    cplx* buf = calloc(6 * np + 2 * nhp, sizeof(cplx));
    if (!buf) { ctx_free(&c); return ORC_ENOMEM; }
    cplx *lF1 = buf, *lP1 = buf + np, *lF = buf + 2 * np, *lP = buf + 3 * np;
    cplx *iF = buf + 4 * np, *iP = buf + 5 * np, *mF = buf + 6 * np, *mP = mF + nhp;
    const cplx *Pi_ = (const cplx*)P_int, *Ph = (const cplx*)P_half;
    const cplx *dPi = (const cplx*)dP_int, *dPh = (const cplx*)dP_half;
    const double dt = c.g.dt;
    double g_r0 = 0.0;
    /* lambda^{N} = E^T dL/dW_N */
    for (int64_t k = nsteps; k >= 1; --k) {
        /* add E^T dL/dW_k to lambda^{step0+k} (held in lF1) */
        const double* gw = gwave + (size_t)(k - 1) * 2 * nth;
        for (int j = 0; j < nth; ++j) {
            cplx g = gw[2 * j] + I * gw[2 * j + 1];
            lF1[(size_t)j * nr + c.g.i_e] += (1.0 - c.g.f_e) * g;
            lF1[(size_t)j * nr + c.g.i_e + 1] += c.g.f_e * g;
        }
        /* step n = step0 + k - 1 maps u^n -> u^{n+1} */
        int64_t n = step0 + k - 1;
        lw_step_adj(&c, lF1, lP1, lF, lP, mF, mP, iF, iP);
        /* source gradients of step n */
        double A = amp_of(amps, n_amps, n);
        double tp = (double)n * dt, tc = tp + 0.5 * dt;
        cplx ep = cexp(-I * (omega * tp + phase0)), ec = cexp(-I * (omega * tc + phase0));
        cplx dep = -I * (domega * tp + dphase0) * ep, dec = -I * (domega * tc + dphase0) * ec;
        double gA = 0.0, gR = 0.0;
        for (int j = 0; j < nth; ++j) {
            for (int i = 0; i < nh; ++i) {
                size_t q = (size_t)j * nh + i;
                cplx mu = mP[q];
                gA += creal(conj(mu) * 0.5 * dt * ep * Ph[q]);
                gR += creal(conj(mu) * 0.5 * dt * A * (dep * Ph[q] + ep * dPh[q]));
            }
            for (int i = 1; i < nr - 1; ++i) {
                size_t q = (size_t)j * nr + i;
                cplx la = iP[q];
                gA += creal(conj(la) * dt * ec * Pi_[q]);
                gR += creal(conj(la) * dt * A * (dec * Pi_[q] + ec * dPi[q]));
            }
        }
        if (grad_amps) grad_amps[k - 1] = gA;
        g_r0 += gR;
        cplx* t;
        t = lF1; lF1 = lF; lF = t;
        t = lP1; lP1 = lP; lP = t;
    }
    if (grad_r0) *grad_r0 = g_r0;
    if (lam0) cplx_to_u(&c, lF1, lP1, lam0);
    free(buf);
    ctx_free(&c);
    return ORC_OK;
}
