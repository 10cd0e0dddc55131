/*
 * lbm_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Restates, node by node and in the paper's order, the algorithm of
 * Klass, Gabbana & Bartel, "Characteristic Boundary Condition for Thermal
 * Lattice Boltzmann Methods" (arXiv 2307.16766):
 *
 *   collide (Eq. bgk) -> stream (Eq. lbe) -> boundary condition -> macros
 *   (Fig. flowchart-lbm-algo), where the boundary condition is the
 *   characteristic analysis of Sec. 3 carried out layer by layer (Sec. 3.3,
 *   Fig. Layer-Multispeed-BC) and integrated with RK4 (Sec. 3.3, "Time
 *   integration"), then imposed as a mesoscopic Dirichlet condition
 *   (equilibrium or Eq. NEEP).  Zero gradient (Eq. zg-bc) and a fixed inflow
 *   equilibrium are the non-characteristic alternatives.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may use
 * this file.  It shares nothing with the CUDA implementation.
 *
 * Readings of the paper taken here:
 *  - Eq. feq-4: the (u.c)^2 (T-1) term uses (xi^2 - 6), not (c^2 - 4): only
 *    then are the Maxwellian moments reproduced (tests/test_oracle_tables.py).
 *  - Eqs. feq-3/feq-4 are the Hermite expansion in xi = c/c_s, u~ = u/c_s.
 *  - Tab. d2q37: c_s and the weights are the solution of the isotropy
 *    conditions (the printed c_s formula does not match the weights).
 *  - Sec. 3.1: the (4,1) entry of S is T~/(4 rho c_s^2).
 *  - Eq. LaplaceU: f^neq = f - f^eq; sigma' = -(1 - 1/(2 tau)) sum c c f^neq.
 *  - Eq. LaplaceT: physical heat flux q = (1 - 1/(2 tau)) 1/2 sum f^neq |c-u|^2 (c-u).
 *  - Sec. 3.3, "Evaluation of viscous terms": the one-sided stencil of the
 *    mesoscopic viscous terms starts M nodes below x_f, at the first node
 *    none of whose populations was streamed from a boundary layer.  At x_f
 *    itself (the literal reading) the moments mix in the Dirichlet-written
 *    layers and the scheme grows on the paper's Sec. 4.2 vortex, where the
 *    paper reports it stable (tests/test_oracle_viscous.py).
 *  - D2Q9 runs isothermal (Sec. 4.4) with the 3x3 system for (rho, u_n, u_t).
 *  - Corners: plain LODI (Eq. PNR) along the outward diagonal at the
 *    innermost corner node, copied to the M x M corner block (Sec. 3.3, 4.4).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "lbm_oracle.h"

#define QMAX 37

typedef struct {
    int q, M, thermal;
    int order;         /* order of the Hermite expansion of f^eq: 2, 3 or 4 */
    double cs2, cs;
    int c[QMAX][2];
    double w[QMAX];
} lattice_t;

/* Append every distinct member of the fully symmetric class (a,b), i.e.
 * (+-a,+-b) and (+-b,+-a), with weight w (Appendix B notation). */
static void add_class(lattice_t* L, int a, int b, double w)
{
    int cand[8][2] = {{a, b}, {-a, b}, {a, -b}, {-a, -b},
                      {b, a}, {-b, a}, {b, -a}, {-b, -a}};
    for (int k = 0; k < 8; k++) {
        int dup = 0;
        for (int i = 0; i < L->q; i++)
            if (L->c[i][0] == cand[k][0] && L->c[i][1] == cand[k][1]) dup = 1;
        if (!dup) {
            L->c[L->q][0] = cand[k][0];
            L->c[L->q][1] = cand[k][1];
            L->w[L->q] = w;
            L->q++;
        }
    }
}

static int make_lattice(int lattice, lattice_t* L)
{
    memset(L, 0, sizeof(*L));
    if (lattice == ORC_D2Q9) {
        /* Appendix B, Tab. d2q9: c_s = 1/sqrt(3). */
        L->M = 1;
        L->thermal = 0;
        L->order = 2;
        L->cs2 = 1.0 / 3.0;
        add_class(L, 0, 0, 4.0 / 9.0);
        add_class(L, 1, 0, 1.0 / 9.0);
        add_class(L, 1, 1, 1.0 / 36.0);
    } else if (lattice == ORC_D2Q37) {
        /* Appendix B, Tab. d2q37 (velocity classes), M = 3.  Weights and c_s
         * to 20 digits: the solution of the isotropy conditions through
         * eighth order; they agree with the printed 14-decimal weights. */
        L->M = 3;
        L->thermal = 1;
        L->order = 4;
        L->cs2 = 0.6979533220196830882384091;
        add_class(L, 0, 0, 0.23315066913235250229);
        add_class(L, 1, 0, 0.10730609154221900241);
        add_class(L, 1, 1, 0.05766785988879488203);
        add_class(L, 2, 0, 0.014208216158450750265);
        add_class(L, 2, 1, 0.0053530490005137752327);
        add_class(L, 2, 2, 0.0010119375926735754754);
        add_class(L, 3, 0, 0.00024530102775771734547);
        add_class(L, 3, 1, 0.0002834142529941982174);
    } else if (lattice == ORC_D2Q17) {
        /* Appendix B, Tab. d2q17: the printed closed-form weights, M = 3,
         * third-order equilibrium (Eq. feq-3).  c_s^2 = 72 / (5 (25 +
         * sqrt 193)) = sum_i w_i c_ix^2 of those weights: the printed c_s
         * formula gives its reciprocal. */
        const double r = sqrt(193.0);
        L->M = 3;
        L->thermal = 1;
        L->order = 3;
        L->cs2 = 72.0 / (5.0 * (25.0 + r));
        add_class(L, 0, 0, (575.0 + 193.0 * r) / 8100.0);
        add_class(L, 1, 0, (3355.0 - 91.0 * r) / 18000.0);
        add_class(L, 1, 1, (655.0 + 17.0 * r) / 27000.0);
        add_class(L, 2, 2, (685.0 - 49.0 * r) / 54000.0);
        add_class(L, 3, 0, (1445.0 - 101.0 * r) / 162000.0);
    } else {
        return -1;
    }
    L->cs = sqrt(L->cs2);
    return 0;
}

int orc_lattice_info(int lattice, int* q, int* M, double* cs2, int* c, double* w)
{
    lattice_t L;
    if (make_lattice(lattice, &L)) return -1;
    if (q) *q = L.q;
    if (M) *M = L.M;
    if (cs2) *cs2 = L.cs2;
    for (int i = 0; i < L.q; i++) {
        if (c) { c[2 * i] = L.c[i][0]; c[2 * i + 1] = L.c[i][1]; }
        if (w) w[i] = L.w[i];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Equilibrium and moments                                                  */
/* ------------------------------------------------------------------------ */

/* Shifted equilibrium g^eq_i = f^eq_i - w_i rho0 at U = (drho, ux, uy, dT).
 * D2Q37: fourth-order Hermite expansion, Eq. feq-4 (built on Eq. feq-3),
 * written in xi = c/c_s, u~ = u/c_s, theta - 1 = dT.
 * D2Q17: the third-order expansion, Eq. feq-3, in the same variables.
 * D2Q9: second-order isothermal expansion (the first bracket of Eq. feq-3
 * with T = 1). */
static void feq_shifted(const lattice_t* L, double rho0, const double U[4], double* g)
{
    double drho = U[0], ux = U[1], uy = U[2];
    double dT = L->thermal ? U[3] : 0.0;
    double rho = rho0 + drho;
    double uu = (ux * ux + uy * uy) / L->cs2;              /* |u~|^2      */
    for (int i = 0; i < L->q; i++) {
        double cx = L->c[i][0], cy = L->c[i][1];
        double xi2 = (cx * cx + cy * cy) / L->cs2;         /* |xi|^2      */
        double xu = (cx * ux + cy * uy) / L->cs2;          /* xi . u~     */
        double h1 = xu;
        double h2 = 0.5 * (xu * xu - uu + dT * (xi2 - 2.0));
        double h3 = 0.0, h4 = 0.0;
        if (L->order >= 3)
            h3 = xu / 6.0 * (xu * xu - 3.0 * uu + 3.0 * dT * (xi2 - 4.0));
        if (L->order >= 4) {
            h4 = (xu * xu * xu * xu - 6.0 * xu * xu * uu + 3.0 * uu * uu
                  + 6.0 * dT * (xu * xu * (xi2 - 6.0) + uu * (4.0 - xi2))
                  + 3.0 * dT * dT * (xi2 * xi2 - 8.0 * xi2 + 8.0)) / 24.0;
        }
        g[i] = L->w[i] * drho + L->w[i] * rho * (h1 + h2 + h3 + h4);
    }
}

/* Eq. macro on shifted populations: rho = rho0 + sum g, rho u = sum g c,
 * sum f |c-u|^2 = 2 rho c_s^2 theta (e = (d/2) T~ with d = 2, T~ = c_s^2 theta),
 * using sum_i w_i c_i = 0 and sum_i w_i |c_i|^2 = 2 c_s^2. */
static void moments_shifted(const lattice_t* L, double rho0, const double* g, double U[4])
{
    double s0 = 0, sx = 0, sy = 0, se = 0;
    for (int i = 0; i < L->q; i++) {
        double cx = L->c[i][0], cy = L->c[i][1];
        s0 += g[i];
        sx += g[i] * cx;
        sy += g[i] * cy;
        se += g[i] * (cx * cx + cy * cy);
    }
    double rho = rho0 + s0;
    double ux = sx / rho, uy = sy / rho;
    U[0] = s0;
    U[1] = ux;
    U[2] = uy;
    U[3] = L->thermal ? (se - rho * (ux * ux + uy * uy) - 2.0 * L->cs2 * s0) / (2.0 * rho * L->cs2)
                      : 0.0;
}

void orc_feq(int lattice, double rho0, const double U[4], double* g)
{
    lattice_t L;
    if (make_lattice(lattice, &L)) return;
    feq_shifted(&L, rho0, U, g);
}

void orc_moments(int lattice, double rho0, const double* g, double U[4])
{
    lattice_t L;
    if (make_lattice(lattice, &L)) return;
    moments_shifted(&L, rho0, g, U);
}

/* Regularised non-equilibrium part (the regularised Dirichlet schemes the
 * paper names for future work, Sec. 5): the projection of g onto the
 * Hermite polynomials of orders 2 and, on the thermal lattices, 3,
 *   g_i <- w_i [ H2_i : a2 / (2 c_s^4) + H3_i : a3 / (6 c_s^6) ],
 *   a_n = sum_i H_n(c_i) g_i,  H2_ab = c_a c_b - c_s^2 d_ab,
 *   H3_abc = c_a c_b c_c - c_s^2 (c_a d_bc + c_b d_ac + c_c d_ab).
 * The quadratures are exact for these products (D2Q9: degree 5 >= 4 for
 * order 2; D2Q17, D2Q37: degree >= 6), so the projection keeps a2 and a3. */
static void regularize(const lattice_t* L, double* g)
{
    const double cs2 = L->cs2;
    double a2[3] = {0, 0, 0}, a3[4] = {0, 0, 0, 0};      /* xx xy yy; xxx xxy xyy yyy */
    for (int i = 0; i < L->q; i++) {
        double cx = L->c[i][0], cy = L->c[i][1];
        a2[0] += (cx * cx - cs2) * g[i];
        a2[1] += cx * cy * g[i];
        a2[2] += (cy * cy - cs2) * g[i];
        a3[0] += (cx * cx * cx - 3.0 * cs2 * cx) * g[i];
        a3[1] += (cx * cx * cy - cs2 * cy) * g[i];
        a3[2] += (cx * cy * cy - cs2 * cx) * g[i];
        a3[3] += (cy * cy * cy - 3.0 * cs2 * cy) * g[i];
    }
    int third = L->order >= 3;
    for (int i = 0; i < L->q; i++) {
        double cx = L->c[i][0], cy = L->c[i][1];
        double h2 = (cx * cx - cs2) * a2[0] + 2.0 * cx * cy * a2[1] + (cy * cy - cs2) * a2[2];
        double h3 = (cx * cx * cx - 3.0 * cs2 * cx) * a3[0] + 3.0 * (cx * cx * cy - cs2 * cy) * a3[1]
                  + 3.0 * (cx * cy * cy - cs2 * cx) * a3[2] + (cy * cy * cy - 3.0 * cs2 * cy) * a3[3];
        g[i] = L->w[i] * (h2 / (2.0 * cs2 * cs2) + (third ? h3 / (6.0 * cs2 * cs2 * cs2) : 0.0));
    }
}

int orc_regularize(int lattice, double* g)
{
    lattice_t L;
    if (make_lattice(lattice, &L)) return -1;
    regularize(&L, g);
    return 0;
}

/* Viscous stress sigma' (Eq. LaplaceU) and heat flux q (Eqs. heatflux,
 * LaplaceT) from the non-equilibrium part f - f^eq of one node.  The
 * equilibrium part of the central third moment vanishes on D2Q37 and D2Q17
 * (their equilibria reproduce the Maxwellian moments through third order),
 * so q is taken from f^neq alone.  Both carry the factor (1 - 1/(2 tau)). */
static void neq_moments(const lattice_t* L, double tau, double rho0, const double* g, double out[5])
{
    double U[4], ge[QMAX];
    moments_shifted(L, rho0, g, U);
    feq_shifted(L, rho0, U, ge);
    double sxx = 0, sxy = 0, syy = 0, qx = 0, qy = 0;
    for (int i = 0; i < L->q; i++) {
        double d = g[i] - ge[i];
        double cx = L->c[i][0], cy = L->c[i][1];
        sxx += cx * cx * d;
        sxy += cx * cy * d;
        syy += cy * cy * d;
        if (L->thermal) {
            double ex = cx - U[1], ey = cy - U[2];
            double e2 = ex * ex + ey * ey;
            qx += 0.5 * d * e2 * ex;
            qy += 0.5 * d * e2 * ey;
        }
    }
    double fac = 1.0 - 1.0 / (2.0 * tau);
    out[0] = -fac * sxx;
    out[1] = -fac * sxy;
    out[2] = -fac * syy;
    out[3] = fac * qx;
    out[4] = fac * qy;
}

/* ------------------------------------------------------------------------ */
/* Characteristic analysis (Sec. 3.1, 3.2)                                  */
/* ------------------------------------------------------------------------ */

static int is_acoustic(int thermal, int i)
{
    return thermal ? (i == 2 || i == 3) : (i == 0 || i == 2);
}

static void char_matrices(const lattice_t* L, double rho0, const double Ul[4],
                          double S[16], double Si[16], double Lam[4])
{
    double rho = rho0 + Ul[0], un = Ul[1];
    double cs2 = L->cs2;
    memset(S, 0, 16 * sizeof(double));
    memset(Si, 0, 16 * sizeof(double));
    if (L->thermal) {
        /* Sec. 3.1: A = S^-1 Lambda S for U = (rho, u_n, u_t, T) with the
         * rescaled temperature T~ = c_s^2 T. */
        double Tt = cs2 * (1.0 + Ul[3]);
        double a = sqrt(Tt / (8.0 * cs2 * cs2));
        double b = sqrt(2.0 * cs2 * cs2 / Tt);
        S[0 * 4 + 0] = -Tt / (2.0 * rho * cs2);  S[0 * 4 + 3] = 0.5;
        S[1 * 4 + 2] = 1.0;
        S[2 * 4 + 0] = Tt / (4.0 * rho * cs2);   S[2 * 4 + 1] = -a;  S[2 * 4 + 3] = 0.25;
        S[3 * 4 + 0] = Tt / (4.0 * rho * cs2);   S[3 * 4 + 1] = a;   S[3 * 4 + 3] = 0.25;
        Si[0 * 4 + 0] = -rho * cs2 / Tt; Si[0 * 4 + 2] = rho * cs2 / Tt; Si[0 * 4 + 3] = rho * cs2 / Tt;
        Si[1 * 4 + 2] = -b;              Si[1 * 4 + 3] = b;
        Si[2 * 4 + 1] = 1.0;
        Si[3 * 4 + 0] = 1.0;             Si[3 * 4 + 2] = 1.0;            Si[3 * 4 + 3] = 1.0;
        double c = sqrt(2.0 * Tt);
        Lam[0] = un; Lam[1] = un; Lam[2] = un - c; Lam[3] = un + c;
    } else {
        /* Isothermal D2Q9 system for (rho, u_n, u_t) with P = c_s^2 rho. */
        double cs = L->cs;
        S[0 * 4 + 0] = 0.5; S[0 * 4 + 1] = -rho / (2.0 * cs);
        S[1 * 4 + 2] = 1.0;
        S[2 * 4 + 0] = 0.5; S[2 * 4 + 1] = rho / (2.0 * cs);
        Si[0 * 4 + 0] = 1.0;       Si[0 * 4 + 2] = 1.0;
        Si[1 * 4 + 0] = -cs / rho; Si[1 * 4 + 2] = cs / rho;
        Si[2 * 4 + 1] = 1.0;
        Lam[0] = un - cs; Lam[1] = un; Lam[2] = un + cs; Lam[3] = 0.0;
    }
}

void orc_char_matrices(int lattice, double rho0, const double Ul[4],
                       double S[16], double Sinv[16], double Lam[4])
{
    lattice_t L;
    if (make_lattice(lattice, &L)) return;
    char_matrices(&L, rho0, Ul, S, Sinv, Lam);
}

static int incoming_mask(const lattice_t* L, double rho0, const double Ul[4])
{
    double S[16], Si[16], Lam[4];
    char_matrices(L, rho0, Ul, S, Si, Lam);
    int n = L->thermal ? 4 : 3, m = 0;
    for (int i = 0; i < n; i++)
        if (Lam[i] < 0.0) m |= 1 << i;   /* wave enters through an outward normal */
    return m;
}

/* Right-hand side of Eq. thermal_LODI_macro_evo (LODI schemes) or
 * Eq. thermal_CBC_macro_evo (CBC schemes), with the incoming amplitudes of
 * Eq. PNR, Eq. LODI-Relax, Eq. CBC-PNR or Eq. CBC-Relax (Tab. CBCs).  The
 * pressure relaxation beta (Z - Z_inf) acts on the incoming acoustic waves. */
static void char_rhs(const lattice_t* L, const orc_params* P, const double Ul[4],
                     const double dUn[4], const double TT[4], const double VV[4],
                     int mask, double dP, int scheme, double k[4])
{
    double S[16], Si[16], Lam[4];
    char_matrices(L, P->rho0, Ul, S, Si, Lam);
    int n = L->thermal ? 4 : 3;
    double Lb[4] = {0, 0, 0, 0};
    for (int i = 0; i < n; i++) {
        double sd = 0, st = 0, sv = 0;
        for (int m = 0; m < n; m++) {
            sd += S[i * 4 + m] * dUn[m];
            st += S[i * 4 + m] * TT[m];
            sv += S[i * 4 + m] * VV[m];
        }
        double Li = Lam[i] * sd;          /* L = Lambda S dU/dn, Eq. thermal_WAV */
        if (!(mask & (1 << i))) {
            Lb[i] = Li;                    /* outgoing: from the bulk           */
            continue;
        }
        double relaxP = is_acoustic(L->thermal, i) ? P->beta_P * dP : 0.0;
        switch (scheme) {
        case ORC_LODI:       Lb[i] = 0.0; break;
        case ORC_LODI_RELAX: Lb[i] = P->alpha_T * (P->t_inf - st) + relaxP; break;
        case ORC_CBC:        Lb[i] = st + sv; break;
        default:             /* Eq. CBC-Relax, with the viscous term relaxed
                                towards 0 at rate alpha_V (0: the paper's) */
                             Lb[i] = st + sv + P->alpha_T * (P->t_inf - st) +
                                     P->alpha_V * (0.0 - sv) + relaxP; break;
        }
    }
    int cbc = (scheme == ORC_CBC || scheme == ORC_CBC_RELAX);
    for (int m = 0; m < 4; m++) k[m] = 0.0;
    for (int m = 0; m < n; m++) {
        double a = 0;
        for (int i = 0; i < n; i++) a += Si[m * 4 + i] * Lb[i];
        k[m] = -a + (cbc ? TT[m] + VV[m] : 0.0);
    }
}

void orc_char_rhs(const orc_params* p, const double Ul[4], const double dUn[4],
                  const double TT[4], const double VV[4], int incoming_mask_,
                  double dP, int scheme, double k[4])
{
    lattice_t L;
    if (make_lattice(p->lattice, &L)) return;
    char_rhs(&L, p, Ul, dUn, TT, VV, incoming_mask_, dP, scheme, k);
}

/* ------------------------------------------------------------------------ */
/* Classical fourth-order Runge-Kutta (Sec. 3.3, "Time integration")        */
/* ------------------------------------------------------------------------ */

typedef void (*rhs_fn)(void* ctx, double s, const double* Y, double* k);

/* One RK4 step of size h.  The stage time fraction s (0, 1/2, 1/2, 1) is
 * passed to F so that bulk data can be interpolated linearly in time. */
static void rk4_step(int n, double* Y, double h, rhs_fn F, void* ctx, double* work)
{
    double* Ys = work;
    double* k = work + n;
    double* acc = work + 2 * n;
    F(ctx, 0.0, Y, k);
    for (int i = 0; i < n; i++) { acc[i] = k[i];        Ys[i] = Y[i] + 0.5 * h * k[i]; }
    F(ctx, 0.5, Ys, k);
    for (int i = 0; i < n; i++) { acc[i] += 2.0 * k[i]; Ys[i] = Y[i] + 0.5 * h * k[i]; }
    F(ctx, 0.5, Ys, k);
    for (int i = 0; i < n; i++) { acc[i] += 2.0 * k[i]; Ys[i] = Y[i] + h * k[i]; }
    F(ctx, 1.0, Ys, k);
    for (int i = 0; i < n; i++) { acc[i] += k[i];       Y[i] += h * acc[i] / 6.0; }
}

static void scalar_linear(void* ctx, double s, const double* Y, double* k)
{
    (void)s;
    k[0] = *(const double*)ctx * Y[0];
}

double orc_rk4_scalar(double lam, double y0, double h, int nsteps)
{
    double y = y0, work[3];
    for (int i = 0; i < nsteps; i++) rk4_step(1, &y, h, scalar_linear, &lam, work);
    return y;
}

/* ------------------------------------------------------------------------ */
/* Simulation                                                               */
/* ------------------------------------------------------------------------ */

enum { K_BULK = 0, K_BAND = 1, K_CORNER = 2 };

/* Outward normal and tangent of each side (W, E, S, N). */
static const int SN[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
static const int ST[4][2] = {{0, 1}, {0, 1}, {1, 0}, {1, 0}};
/* Outward diagonal of each corner (SW, SE, NW, NE). */
static const int CD[4][2] = {{-1, -1}, {1, -1}, {-1, 1}, {1, 1}};

struct orc_sim {
    orc_params P;
    lattice_t L;
    int nx, ny, q, M, perx, pery, corner_kind;
    double *g, *gpost, *gnew;    /* [ny*nx*q] shifted populations           */
    double *Ut, *Ut1;            /* [ny*nx*4] macros at t and t+1           */
    double *Ub;                  /* [ny*nx*4] characteristic boundary state */
    double *W;                   /* [ny*nx*4] RK4 stage field               */
    unsigned char* kind;         /* K_BULK / K_BAND / K_CORNER              */
    signed char* where;          /* side of a band node, corner id          */
    int ncbc;                    /* unknowns of the boundary ODE            */
    int *u_node, *u_side, *u_j, *u_p;
    double *V;                   /* frozen viscous vectors [ncbc*4]         */
    int* mask;                   /* frozen incoming masks                   */
    double *Y, *work;
    long steps;
};

static inline int wrapi(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

/* Node index at (x, y), wrapping periodic axes; -1 outside the grid. */
static int node_at(const orc_sim* s, int x, int y)
{
    if (s->perx) x = wrapi(x, s->nx);
    else if (x < 0 || x >= s->nx) return -1;
    if (s->pery) y = wrapi(y, s->ny);
    else if (y < 0 || y >= s->ny) return -1;
    return y * s->nx + x;
}

/* Layer-0 node x_f of side sd at tangential position p (Fig. Layer-Multispeed-BC). */
static void xf_of(const orc_sim* s, int sd, int p, int* x, int* y)
{
    int M = s->M;
    switch (sd) {
    case 0: *x = M; *y = p; break;
    case 1: *x = s->nx - 1 - M; *y = p; break;
    case 2: *x = p; *y = M; break;
    default: *x = p; *y = s->ny - 1 - M; break;
    }
}

static void corner_node(const orc_sim* s, int cid, int* x, int* y)
{
    int M = s->M;
    *x = CD[cid][0] < 0 ? M - 1 : s->nx - M;
    *y = CD[cid][1] < 0 ? M - 1 : s->ny - M;
}

/* Lab <-> local frame of an orthonormal pair (n, t). */
static void to_local(const double* U, const double n[2], const double t[2], double* Ul)
{
    Ul[0] = U[0];
    Ul[1] = U[1] * n[0] + U[2] * n[1];
    Ul[2] = U[1] * t[0] + U[2] * t[1];
    Ul[3] = U[3];
}

static void to_lab(const double* Ul, const double n[2], const double t[2], double* U)
{
    U[0] = Ul[0];
    U[1] = Ul[1] * n[0] + Ul[2] * t[0];
    U[2] = Ul[1] * n[1] + Ul[2] * t[1];
    U[3] = Ul[3];
}

static void side_frame(int sd, double n[2], double t[2])
{
    n[0] = SN[sd][0]; n[1] = SN[sd][1];
    t[0] = ST[sd][0]; t[1] = ST[sd][1];
}

static void corner_frame(int cid, double n[2], double t[2])
{
    double r = 1.0 / sqrt(2.0);
    n[0] = CD[cid][0] * r; n[1] = CD[cid][1] * r;
    t[0] = -n[1];          t[1] = n[0];
}

static int validate(const orc_params* p, const lattice_t* L)
{
    if (p->nx < 1 || p->ny < 1 || !(p->tau > 0.5)) return -1;
    if ((p->side[0] == ORC_PERIODIC) != (p->side[1] == ORC_PERIODIC)) return -1;
    if ((p->side[2] == ORC_PERIODIC) != (p->side[3] == ORC_PERIODIC)) return -1;
    if (p->viscous < 0 || p->viscous > 2 || p->dirichlet < 0 || p->dirichlet > 2) return -1;
    for (int sd = 0; sd < 4; sd++) {
        if (p->side[sd] < 0 || p->side[sd] > 3) return -1;
        if (p->scheme[sd] < 0 || p->scheme[sd] > 3) return -1;
    }
    if (p->side[0] != ORC_PERIODIC && p->nx < 2 * L->M + 3) return -1;
    if (p->side[2] != ORC_PERIODIC && p->ny < 2 * L->M + 3) return -1;
    if (p->viscous == ORC_VIS_MESO) {
        /* the mesoscopic stencil's deepest node, x_f - (d0 + 2) n, must be a
         * bulk node */
        int d0 = p->meso_depth < 0 ? L->M : p->meso_depth;
        int need = 2 * L->M + 3 + d0;
        if ((p->side[0] == ORC_SIDE_CBC || p->side[1] == ORC_SIDE_CBC) && p->nx < need) return -1;
        if ((p->side[2] == ORC_SIDE_CBC || p->side[3] == ORC_SIDE_CBC) && p->ny < need) return -1;
    }
    if (p->side[0] != ORC_PERIODIC && p->side[2] != ORC_PERIODIC) {
        int ncbc = 0;
        for (int sd = 0; sd < 4; sd++) ncbc += p->side[sd] == ORC_SIDE_CBC;
        if (ncbc != 0 && ncbc != 4) return -1;  /* corners join like sides only */
    }
    return 0;
}

orc_sim* orc_create(const orc_params* p)
{
    lattice_t L;
    if (make_lattice(p->lattice, &L)) return NULL;
    if (validate(p, &L)) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->P = *p;
    s->L = L;
    s->nx = p->nx;
    s->ny = p->ny;
    s->q = L.q;
    s->M = L.M;
    s->perx = p->side[0] == ORC_PERIODIC;
    s->pery = p->side[2] == ORC_PERIODIC;
    size_t N = (size_t)s->nx * s->ny;
    s->g = (double*)calloc(N * s->q, sizeof(double));
    s->gpost = (double*)calloc(N * s->q, sizeof(double));
    s->gnew = (double*)calloc(N * s->q, sizeof(double));
    s->Ut = (double*)calloc(N * 4, sizeof(double));
    s->Ut1 = (double*)calloc(N * 4, sizeof(double));
    s->Ub = (double*)calloc(N * 4, sizeof(double));
    s->W = (double*)calloc(N * 4, sizeof(double));
    s->kind = (unsigned char*)calloc(N, 1);
    s->where = (signed char*)calloc(N, 1);

    int M = s->M;
    for (int y = 0; y < s->ny; y++)
        for (int x = 0; x < s->nx; x++) {
            int inW = !s->perx && x < M, inE = !s->perx && x >= s->nx - M;
            int inS = !s->pery && y < M, inN = !s->pery && y >= s->ny - M;
            int n = y * s->nx + x;
            if ((inW || inE) && (inS || inN)) {
                s->kind[n] = K_CORNER;
                s->where[n] = (signed char)((inE ? 1 : 0) + (inN ? 2 : 0));
            } else if (inW || inE || inS || inN) {
                s->kind[n] = K_BAND;
                s->where[n] = (signed char)(inW ? 0 : inE ? 1 : inS ? 2 : 3);
            }
        }
    /* Corner kind: characteristic only between characteristic sides. */
    s->corner_kind = ORC_SIDE_ZG;
    if (!s->perx && !s->pery) {
        if (p->side[0] == ORC_SIDE_CBC) s->corner_kind = ORC_SIDE_CBC;
        else if (p->side[0] == ORC_SIDE_INFLOW || p->side[1] == ORC_SIDE_INFLOW ||
                 p->side[2] == ORC_SIDE_INFLOW || p->side[3] == ORC_SIDE_INFLOW)
            s->corner_kind = ORC_SIDE_INFLOW;
    }

    /* Unknowns of the boundary ODE: every layer j = 1..M of every CBC side
     * position, then the CBC corners (one innermost node each). */
    int cap = 0;
    for (int sd = 0; sd < 4; sd++)
        if (p->side[sd] == ORC_SIDE_CBC) cap += M * (sd < 2 ? s->ny : s->nx);
    cap += 4;
    s->u_node = (int*)calloc(cap, sizeof(int));
    s->u_side = (int*)calloc(cap, sizeof(int));
    s->u_j = (int*)calloc(cap, sizeof(int));
    s->u_p = (int*)calloc(cap, sizeof(int));
    int nu = 0;
    for (int sd = 0; sd < 4; sd++) {
        if (p->side[sd] != ORC_SIDE_CBC) continue;
        int len = sd < 2 ? s->ny : s->nx;
        int tper = sd < 2 ? s->pery : s->perx;
        int lo = tper ? 0 : M, hi = tper ? len - 1 : len - 1 - M;
        for (int pp = lo; pp <= hi; pp++)
            for (int j = 1; j <= M; j++) {
                int x, y;
                xf_of(s, sd, pp, &x, &y);
                x += j * SN[sd][0];
                y += j * SN[sd][1];
                s->u_node[nu] = y * s->nx + x;
                s->u_side[nu] = sd;
                s->u_j[nu] = j;
                s->u_p[nu] = pp;
                nu++;
            }
    }
    if (s->corner_kind == ORC_SIDE_CBC)
        for (int cid = 0; cid < 4; cid++) {
            int x, y;
            corner_node(s, cid, &x, &y);
            s->u_node[nu] = y * s->nx + x;
            s->u_side[nu] = 4 + cid;
            s->u_j[nu] = 0;
            s->u_p[nu] = 0;
            nu++;
        }
    s->ncbc = nu;
    s->V = (double*)calloc((size_t)4 * (nu + 1), sizeof(double));
    s->mask = (int*)calloc(nu + 1, sizeof(int));
    s->Y = (double*)calloc((size_t)4 * (nu + 1), sizeof(double));
    s->work = (double*)calloc((size_t)12 * (nu + 1), sizeof(double));
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    free(s->g); free(s->gpost); free(s->gnew);
    free(s->Ut); free(s->Ut1); free(s->Ub); free(s->W);
    free(s->kind); free(s->where);
    free(s->u_node); free(s->u_side); free(s->u_j); free(s->u_p);
    free(s->V); free(s->mask); free(s->Y); free(s->work);
    free(s);
}

/* Set the whole M x M block of corner cid to the 4-vector U in array A. */
static void fill_corner_block(const orc_sim* s, int cid, const double* U, double* A)
{
    for (int a = 0; a < s->M; a++)
        for (int b = 0; b < s->M; b++) {
            int x = CD[cid][0] < 0 ? a : s->nx - 1 - a;
            int y = CD[cid][1] < 0 ? b : s->ny - 1 - b;
            memcpy(A + 4 * (y * s->nx + x), U, 4 * sizeof(double));
        }
}

void orc_init(orc_sim* s, const double* rho, const double* ux, const double* uy, const double* T)
{
    size_t N = (size_t)s->nx * s->ny;
    for (size_t n = 0; n < N; n++) {
        double U[4] = {rho[n] - s->P.rho0, ux[n], uy[n], s->L.thermal ? T[n] - 1.0 : 0.0};
        feq_shifted(&s->L, s->P.rho0, U, s->g + n * s->q);
        memcpy(s->Ub + 4 * n, U, sizeof(U));
    }
    if (s->corner_kind == ORC_SIDE_CBC)
        for (int cid = 0; cid < 4; cid++) {
            int x, y;
            corner_node(s, cid, &x, &y);
            double U[4];
            memcpy(U, s->Ub + 4 * (y * s->nx + x), sizeof(U));
            fill_corner_block(s, cid, U, s->Ub);
        }
    s->steps = 0;
}

/* ---- viscous terms ---------------------------------------------------- */

static int is_bulk(const orc_sim* s, int n) { return n >= 0 && s->kind[n] == K_BULK; }

/* Mesoscopic viscous vector of side sd with its stencil starting at node
 * (x, y), from the pre-collision populations of time t (Sec. 3.3,
 * "Evaluation of viscous terms"): normal derivatives one-sided into the bulk
 * (Eq. FD-dx-bw through (x, y), (x, y) - n, (x, y) - 2n), tangential
 * derivatives central (Eq. FD-dx-center), one-sided inward where the
 * tangential neighbour is itself a boundary node. */
static void vis_meso(const orc_sim* s, int sd, int x, int y, double V[4])
{
    double n[2], t[2];
    side_frame(sd, n, t);
    int nn[2] = {SN[sd][0], SN[sd][1]}, tt[2] = {ST[sd][0], ST[sd][1]};
    /* stencil nodes: 0 = x_f, 1 = x_f - n, 2 = x_f - 2n, 3 = x_f + t,
     * 4 = x_f - t, 5 = x_f + 2t, 6 = x_f - 2t */
    int nd[7];
    nd[0] = node_at(s, x, y);
    nd[1] = node_at(s, x - nn[0], y - nn[1]);
    nd[2] = node_at(s, x - 2 * nn[0], y - 2 * nn[1]);
    nd[3] = node_at(s, x + tt[0], y + tt[1]);
    nd[4] = node_at(s, x - tt[0], y - tt[1]);
    nd[5] = node_at(s, x + 2 * tt[0], y + 2 * tt[1]);
    nd[6] = node_at(s, x - 2 * tt[0], y - 2 * tt[1]);
    int tmode = 0;                       /* 0 central, +1 backward, -1 forward */
    if (!is_bulk(s, nd[3])) tmode = 1;
    else if (!is_bulk(s, nd[4])) tmode = -1;

    /* h[k][*] = (s_nn, s_nt, s_tt, q_n, q_t, u_n, u_t) at stencil node k */
    double h[7][7];
    for (int k = 0; k < 7; k++) {
        if (nd[k] < 0 || (k >= 3 && !((tmode == 0 && (k == 3 || k == 4)) ||
                                      (tmode == 1 && (k == 4 || k == 6)) ||
                                      (tmode == -1 && (k == 3 || k == 5)))))
            continue;
        const double* gk = s->g + (size_t)nd[k] * s->q;
        double o[5], U[4];
        neq_moments(&s->L, s->P.tau, s->P.rho0, gk, o);
        moments_shifted(&s->L, s->P.rho0, gk, U);
        double sig[2][2] = {{o[0], o[1]}, {o[1], o[2]}};
        double sn[2] = {sig[0][0] * n[0] + sig[0][1] * n[1], sig[1][0] * n[0] + sig[1][1] * n[1]};
        double st[2] = {sig[0][0] * t[0] + sig[0][1] * t[1], sig[1][0] * t[0] + sig[1][1] * t[1]};
        h[k][0] = n[0] * sn[0] + n[1] * sn[1];
        h[k][1] = t[0] * sn[0] + t[1] * sn[1];
        h[k][2] = t[0] * st[0] + t[1] * st[1];
        h[k][3] = o[3] * n[0] + o[4] * n[1];
        h[k][4] = o[3] * t[0] + o[4] * t[1];
        h[k][5] = U[1] * n[0] + U[2] * n[1];
        h[k][6] = U[1] * t[0] + U[2] * t[1];
    }
    double dn[7], dt[7];
    for (int m = 0; m < 7; m++) {
        dn[m] = 0.5 * (3.0 * h[0][m] - 4.0 * h[1][m] + h[2][m]);
        if (tmode == 0) dt[m] = 0.5 * (h[3][m] - h[4][m]);
        else if (tmode == 1) dt[m] = 0.5 * (3.0 * h[0][m] - 4.0 * h[4][m] + h[6][m]);
        else dt[m] = -0.5 * (3.0 * h[0][m] - 4.0 * h[3][m] + h[5][m]);
    }
    double U0[4];
    moments_shifted(&s->L, s->P.rho0, s->g + (size_t)nd[0] * s->q, U0);
    double rho = s->P.rho0 + U0[0];
    V[0] = 0.0;
    V[1] = (dn[0] + dt[1]) / rho;        /* (1/rho) d_j sigma'_jn */
    V[2] = (dn[1] + dt[2]) / rho;        /* (1/rho) d_j sigma'_jt */
    V[3] = 0.0;
    if (s->L.thermal) {
        double cs2 = s->L.cs2, nu = (s->P.tau - 0.5) * cs2;
        double heat = (dn[5] - dt[6]) * (dn[5] - dt[6]) + (dn[6] + dt[5]) * (dn[6] + dt[5]);
        V[3] = -(dn[3] + dt[4]) / (rho * cs2) + nu / cs2 * heat;
    }
}

void orc_vis_meso_at(const orc_sim* s, int side, int x, int y, double V[4])
{
    vis_meso(s, side, x, y, V);
}

void orc_neq_moments(const orc_sim* s, int x, int y, double out[5])
{
    int n = node_at(s, x, y);
    neq_moments(&s->L, s->P.tau, s->P.rho0, s->g + (size_t)n * s->q, out);
}

/* -FD viscous vector at layer j of side sd (Sec. 4.2, "Treatment of viscous
 * terms"): 4-point one-sided second derivative at j = M, 3-point central for
 * j < M and along the side; field W holds the macros of time t. */
static void vis_fd(const orc_sim* s, int sd, int j, int p, const double* W, double V[4])
{
    double n[2], t[2];
    side_frame(sd, n, t);
    int x, y;
    xf_of(s, sd, p, &x, &y);
    x += j * SN[sd][0];
    y += j * SN[sd][1];
    int nn0 = SN[sd][0], nn1 = SN[sd][1], t0 = ST[sd][0], t1 = ST[sd][1];
    double U[4], Um1[4], Um2[4], Um3[4], Up1[4] = {0, 0, 0, 0}, Utp[4], Utm[4];
    to_local(W + 4 * node_at(s, x, y), n, t, U);
    to_local(W + 4 * node_at(s, x - nn0, y - nn1), n, t, Um1);
    to_local(W + 4 * node_at(s, x - 2 * nn0, y - 2 * nn1), n, t, Um2);
    to_local(W + 4 * node_at(s, x - 3 * nn0, y - 3 * nn1), n, t, Um3);
    if (j < s->M) to_local(W + 4 * node_at(s, x + nn0, y + nn1), n, t, Up1);
    to_local(W + 4 * node_at(s, x + t0, y + t1), n, t, Utp);
    to_local(W + 4 * node_at(s, x - t0, y - t1), n, t, Utm);
    double dnn[4], dtt[4], d1n[4], d1t[4];
    for (int m = 0; m < 4; m++) {
        if (j == s->M) {
            dnn[m] = 2.0 * U[m] - 5.0 * Um1[m] + 4.0 * Um2[m] - Um3[m];
            d1n[m] = 0.5 * (3.0 * U[m] - 4.0 * Um1[m] + Um2[m]);
        } else {
            dnn[m] = Up1[m] - 2.0 * U[m] + Um1[m];
            d1n[m] = 0.5 * (Up1[m] - Um1[m]);
        }
        dtt[m] = Utp[m] - 2.0 * U[m] + Utm[m];
        d1t[m] = 0.5 * (Utp[m] - Utm[m]);
    }
    double nu = (s->P.tau - 0.5) * s->L.cs2;
    V[0] = 0.0;
    V[1] = nu * (dnn[1] + dtt[1]);
    V[2] = nu * (dnn[2] + dtt[2]);
    V[3] = 0.0;
    if (s->L.thermal) {
        double heat = (d1n[1] - d1t[2]) * (d1n[1] - d1t[2]) + (d1n[2] + d1t[1]) * (d1n[2] + d1t[1]);
        V[3] = 2.0 * nu * (dnn[3] + dtt[3]) + nu / s->L.cs2 * heat;
    }
}

/* ---- boundary ODE right-hand side ------------------------------------- */

/* Pressure excess P - P_inf of a lab state, P = rho c_s^2 T (Sec. 2). */
static double pressure_excess(const orc_sim* s, int sd, const double* U)
{
    double cs2 = s->L.cs2, rho0 = s->P.rho0;
    double rhoT_dev = U[0] + (s->L.thermal ? rho0 * U[3] + U[0] * U[3] : 0.0);
    return cs2 * rhoT_dev - (s->P.p_inf[sd] - cs2 * rho0);
}

static void fill_stage_field(orc_sim* s, double frac, const double* Y)
{
    size_t N = (size_t)s->nx * s->ny;
    for (size_t n = 0; n < N; n++)
        for (int m = 0; m < 4; m++)
            s->W[4 * n + m] = (1.0 - frac) * s->Ut[4 * n + m] + frac * s->Ut1[4 * n + m];
    for (int u = 0; u < s->ncbc; u++) {
        if (s->u_side[u] < 4) memcpy(s->W + 4 * (size_t)s->u_node[u], Y + 4 * u, 4 * sizeof(double));
        else fill_corner_block(s, s->u_side[u] - 4, Y + 4 * u, s->W);
    }
}

/* Corner cid (Sec. 3.3, Fig. Layer-Multispeed-BC): LODI (Eq. PNR) along the
 * outward diagonal n at the innermost corner node, the normal derivative by
 * the one-sided difference of Eq. FD-dx-bw through the node (lab state Uc)
 * and the two diagonal nodes inward (U1 = one diagonal step in, U2 = two),
 * whose spacing is sqrt(2).  k: lab-frame right-hand side. */
static void corner_rhs(const lattice_t* L, const orc_params* P, int cid, const double* Uc,
                       const double* U1lab, const double* U2lab, int mask, double k[4])
{
    double n[2], t[2];
    corner_frame(cid, n, t);
    double U[4], U1[4], U2[4], dUn[4], kl[4], zero[4] = {0, 0, 0, 0};
    to_local(Uc, n, t, U);
    to_local(U1lab, n, t, U1);
    to_local(U2lab, n, t, U2);
    for (int m = 0; m < 4; m++) dUn[m] = (3.0 * U[m] - 4.0 * U1[m] + U2[m]) / (2.0 * sqrt(2.0));
    char_rhs(L, P, U, dUn, zero, zero, mask, 0.0, ORC_LODI, kl);
    to_lab(kl, n, t, k);
}

int orc_corner_rhs(const orc_params* p, int cid, const double Uc[4], const double U1[4],
                   const double U2[4], double k[4])
{
    lattice_t L;
    if (make_lattice(p->lattice, &L) || cid < 0 || cid > 3) return -1;
    double n[2], t[2], Ul[4];
    corner_frame(cid, n, t);
    to_local(Uc, n, t, Ul);
    corner_rhs(&L, p, cid, Uc, U1, U2, incoming_mask(&L, p->rho0, Ul), k);
    return 0;
}

/* Right-hand side at one characteristic unknown from the stage field W. */
static void unknown_rhs(const orc_sim* s, int u, double k[4])
{
    const double* W = s->W;
    int sd = s->u_side[u];
    if (sd >= 4) {
        int cid = sd - 4, node = s->u_node[u], x = node % s->nx, y = node / s->nx;
        corner_rhs(&s->L, &s->P, cid, W + 4 * node,
                   W + 4 * node_at(s, x - CD[cid][0], y - CD[cid][1]),
                   W + 4 * node_at(s, x - 2 * CD[cid][0], y - 2 * CD[cid][1]), s->mask[u], k);
        return;
    }
    double n[2], t[2];
    side_frame(sd, n, t);
    int j = s->u_j[u], node = s->u_node[u], x = node % s->nx, y = node / s->nx;
    int nn0 = SN[sd][0], nn1 = SN[sd][1], t0 = ST[sd][0], t1 = ST[sd][1];
    double U[4], A[4], B[4], dUn[4];
    to_local(W + 4 * node, n, t, U);
    if (j == s->M) {
        /* Eq. FD-dx-bw at the outermost layer */
        to_local(W + 4 * node_at(s, x - nn0, y - nn1), n, t, A);
        to_local(W + 4 * node_at(s, x - 2 * nn0, y - 2 * nn1), n, t, B);
        for (int m = 0; m < 4; m++) dUn[m] = 0.5 * (3.0 * U[m] - 4.0 * A[m] + B[m]);
    } else {
        /* Eq. FD-dx-center at inner layers */
        to_local(W + 4 * node_at(s, x + nn0, y + nn1), n, t, A);
        to_local(W + 4 * node_at(s, x - nn0, y - nn1), n, t, B);
        for (int m = 0; m < 4; m++) dUn[m] = 0.5 * (A[m] - B[m]);
    }
    /* Transversal vector (Sec. 3.1) with central differences along the side. */
    double Up[4], Um[4];
    to_local(W + 4 * node_at(s, x + t0, y + t1), n, t, Up);
    to_local(W + 4 * node_at(s, x - t0, y - t1), n, t, Um);
    double rho0 = s->P.rho0, cs2 = s->L.cs2, rho = rho0 + U[0], ut = U[2];
    double rp = rho0 + Up[0], rm = rho0 + Um[0];
    double d_rhout = 0.5 * (rp * Up[2] - rm * Um[2]);
    double d_un = 0.5 * (Up[1] - Um[1]);
    double d_ut = 0.5 * (Up[2] - Um[2]);
    double TT[4];
    if (s->L.thermal) {
        double d_rhoT = 0.5 * ((Up[0] + rho0 * Up[3] + Up[0] * Up[3]) - (Um[0] + rho0 * Um[3] + Um[0] * Um[3]));
        double d_Tut = 0.5 * ((1.0 + Up[3]) * Up[2] - (1.0 + Um[3]) * Um[2]);
        TT[0] = -d_rhout;
        TT[1] = -ut * d_un;
        TT[2] = -(cs2 / rho) * d_rhoT - ut * d_ut;
        TT[3] = -d_Tut;
    } else {
        double d_rho = 0.5 * (Up[0] - Um[0]);
        TT[0] = -d_rhout;
        TT[1] = -ut * d_un;
        TT[2] = -(cs2 / rho) * d_rho - ut * d_ut;
        TT[3] = 0.0;
    }
    double Ulab[4];
    memcpy(Ulab, W + 4 * node, sizeof(Ulab));
    double dP = pressure_excess(s, sd, Ulab);
    double kl[4];
    char_rhs(&s->L, &s->P, U, dUn, TT, s->V + 4 * u, s->mask[u], dP, s->P.scheme[sd], kl);
    to_lab(kl, n, t, k);
}

static void band_rhs(void* ctx, double frac, const double* Y, double* k)
{
    orc_sim* s = (orc_sim*)ctx;
    fill_stage_field(s, frac, Y);
    for (int u = 0; u < s->ncbc; u++) unknown_rhs(s, u, k + 4 * u);
}

/* ---- one time step ----------------------------------------------------- */

static void step_once(orc_sim* s)
{
    const int q = s->q, nx = s->nx, ny = s->ny;
    const lattice_t* L = &s->L;
    const double tau = s->P.tau, rho0 = s->P.rho0;

    /* Collide every node, boundary nodes included (Eq. bgk). */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t n = (size_t)y * nx + x;
            double ge[QMAX];
            const double* g = s->g + n * q;
            double* gp = s->gpost + n * q;
            moments_shifted(L, rho0, g, s->Ut + 4 * n);
            feq_shifted(L, rho0, s->Ut + 4 * n, ge);
            for (int i = 0; i < q; i++) gp[i] = g[i] - (g[i] - ge[i]) / tau;
        }

    /* Stream into every bulk node (Eq. lbe), wrapping periodic axes. */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t n = (size_t)y * nx + x;
            if (s->kind[n] != K_BULK) continue;
            for (int i = 0; i < q; i++) {
                int src = node_at(s, x - L->c[i][0], y - L->c[i][1]);
                s->gnew[n * q + i] = s->gpost[(size_t)src * q + i];
            }
            moments_shifted(L, rho0, s->gnew + n * q, s->Ut1 + 4 * n);
        }

    /* Non-characteristic boundary nodes: zero gradient (Eq. zg-bc) copies x_f;
     * inflow imposes the equilibrium of the inflow state. */
    double Uin[4] = {s->P.inflow[0] - rho0, s->P.inflow[1], s->P.inflow[2],
                     L->thermal ? s->P.inflow[3] - 1.0 : 0.0};
    double gin[QMAX];
    feq_shifted(L, rho0, Uin, gin);
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t n = (size_t)y * nx + x;
            int kind = s->kind[n];
            if (kind == K_BULK) continue;
            int bc;
            int src = -1;
            if (kind == K_BAND) {
                int sd = s->where[n];
                bc = s->P.side[sd];
                int j = (sd == 0) ? s->M - x : (sd == 1) ? x - (nx - 1 - s->M)
                       : (sd == 2) ? s->M - y : y - (ny - 1 - s->M);
                src = node_at(s, x - j * SN[sd][0], y - j * SN[sd][1]);
            } else {
                bc = s->corner_kind;
                int cid = s->where[n], cx, cy;
                corner_node(s, cid, &cx, &cy);
                src = node_at(s, cx - CD[cid][0], cy - CD[cid][1]);
            }
            if (bc == ORC_SIDE_ZG) memcpy(s->gnew + n * q, s->gnew + (size_t)src * q, q * sizeof(double));
            else if (bc == ORC_SIDE_INFLOW) memcpy(s->gnew + n * q, gin, q * sizeof(double));
            else continue;
            moments_shifted(L, rho0, s->gnew + n * q, s->Ut1 + 4 * n);
        }

    if (s->ncbc > 0) {
        /* Frozen at time t: viscous vectors and incoming-wave masks (the sign
         * of Lambda at t+1 is taken from t, Sec. 3.2). */
        for (int u = 0; u < s->ncbc; u++) memcpy(s->Y + 4 * u, s->Ub + 4 * (size_t)s->u_node[u], 4 * sizeof(double));
        fill_stage_field(s, 0.0, s->Y);
        for (int u = 0; u < s->ncbc; u++) {
            int sd = s->u_side[u];
            double n[2], t[2], Ul[4];
            if (sd >= 4) {
                corner_frame(sd - 4, n, t);
                memset(s->V + 4 * u, 0, 4 * sizeof(double));
            } else {
                side_frame(sd, n, t);
                if (s->P.viscous == ORC_VIS_OFF) {
                    memset(s->V + 4 * u, 0, 4 * sizeof(double));
                } else if (s->P.viscous == ORC_VIS_FD) {
                    vis_fd(s, sd, s->u_j[u], s->u_p[u], s->W, s->V + 4 * u);
                } else {
                    /* stencil start: M nodes below x_f (see the readings) */
                    int x, y, d0 = s->P.meso_depth < 0 ? s->M : s->P.meso_depth;
                    xf_of(s, sd, s->u_p[u], &x, &y);
                    vis_meso(s, sd, x - d0 * SN[sd][0], y - d0 * SN[sd][1], s->V + 4 * u);
                }
            }
            to_local(s->Y + 4 * u, n, t, Ul);
            s->mask[u] = incoming_mask(L, rho0, Ul);
        }
        /* RK4 over all layers and corners at once. */
        rk4_step(4 * s->ncbc, s->Y, 1.0, band_rhs, s, s->work);

        /* Mesoscopic Dirichlet condition: equilibrium (+ NEEP, or its
         * regularised form). */
        for (int u = 0; u < s->ncbc; u++) {
            int sd = s->u_side[u];
            const double* Unew = s->Y + 4 * u;
            double ge[QMAX], gf[QMAX];
            feq_shifted(L, rho0, Unew, ge);
            int src;
            int node = s->u_node[u], x = node % nx, y = node / nx;
            if (sd < 4) src = node_at(s, x - s->u_j[u] * SN[sd][0], y - s->u_j[u] * SN[sd][1]);
            else src = node_at(s, x - CD[sd - 4][0], y - CD[sd - 4][1]);
            if (s->P.dirichlet >= 1) {
                double gn[QMAX];
                feq_shifted(L, rho0, s->Ut1 + 4 * (size_t)src, gf);
                for (int i = 0; i < q; i++) gn[i] = s->gnew[(size_t)src * q + i] - gf[i];
                if (s->P.dirichlet == 2) regularize(L, gn);
                for (int i = 0; i < q; i++) ge[i] += gn[i];
            }
            if (sd < 4) {
                memcpy(s->gnew + (size_t)node * q, ge, q * sizeof(double));
                memcpy(s->Ub + 4 * (size_t)node, Unew, 4 * sizeof(double));
            } else {
                int cid = sd - 4;
                for (int a = 0; a < s->M; a++)
                    for (int b = 0; b < s->M; b++) {
                        int xx = CD[cid][0] < 0 ? a : nx - 1 - a;
                        int yy = CD[cid][1] < 0 ? b : ny - 1 - b;
                        memcpy(s->gnew + (size_t)(yy * nx + xx) * q, ge, q * sizeof(double));
                    }
                fill_corner_block(s, cid, Unew, s->Ub);
            }
        }
    }

    double* tmp = s->g;
    s->g = s->gnew;
    s->gnew = tmp;
    s->steps++;
}

void orc_step(orc_sim* s, int n)
{
    for (int i = 0; i < n; i++) step_once(s);
}

void orc_macros(const orc_sim* s, double* rho, double* ux, double* uy, double* T)
{
    size_t N = (size_t)s->nx * s->ny;
    for (size_t n = 0; n < N; n++) {
        double U[4];
        moments_shifted(&s->L, s->P.rho0, s->g + n * s->q, U);
        rho[n] = s->P.rho0 + U[0];
        ux[n] = U[1];
        uy[n] = U[2];
        T[n] = 1.0 + U[3];
    }
}

void orc_populations(const orc_sim* s, double* g)
{
    memcpy(g, s->g, (size_t)s->nx * s->ny * s->q * sizeof(double));
}

void orc_boundary_state(const orc_sim* s, double* Ub)
{
    memcpy(Ub, s->Ub, (size_t)s->nx * s->ny * 4 * sizeof(double));
}

long orc_steps_done(const orc_sim* s) { return s->steps; }

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following steps (n >= 1); returns the count now in use.
 * The result of a step does not depend on it (rows are independent). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return orc_threads();
}
