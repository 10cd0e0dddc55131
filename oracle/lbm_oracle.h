/*
 * lbm_oracle.h -- plain FP64 CPU oracle for the thermal lattice Boltzmann
 * method with the layer-wise characteristic boundary condition of
 * Klass, Gabbana & Bartel, "Characteristic Boundary Condition for Thermal
 * Lattice Boltzmann Methods" (arXiv 2307.16766).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this code; only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py use it.  It shares no code,
 * header, table or constant with the CUDA implementation.
 *
 * Conventions (all FP64):
 *   - populations are held shifted, g_i = f_i - w_i rho0 (an exact change of
 *     variables: Eq. lbe and Eq. bgk are linear in f and f^eq(rho0,0,1) =
 *     w rho0), which keeps small perturbations free of cancellation;
 *   - macroscopic state is carried as deviations U = (drho, ux, uy, dT) with
 *     rho = rho0 + drho and the dimensionless temperature theta = 1 + dT
 *     (Sec. 3.1: T~ = c_s^2 T with reference temperature T0 = 1);
 *   - grid arrays are row-major [ny][nx] with x fastest;
 *   - sides are numbered W(-x)=0, E(+x)=1, S(-y)=2, N(+y)=3.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_D2Q9 = 0, ORC_D2Q37 = 1, ORC_D2Q17 = 2 };
enum { ORC_PERIODIC = 0, ORC_SIDE_CBC = 1, ORC_SIDE_INFLOW = 2, ORC_SIDE_ZG = 3 };
enum { ORC_LODI = 0, ORC_LODI_RELAX = 1, ORC_CBC = 2, ORC_CBC_RELAX = 3 };
enum { ORC_VIS_MESO = 0, ORC_VIS_FD = 1, ORC_VIS_OFF = 2 };

typedef struct {
    int lattice;       /* ORC_D2Q9 (isothermal), ORC_D2Q37 or ORC_D2Q17 (thermal) */
    int nx, ny;        /* grid size                                            */
    double tau;        /* BGK relaxation time, Eq. bgk                         */
    double rho0;       /* reference density of the population shift            */
    int side[4];       /* kind of each side (W,E,S,N)                          */
    int scheme[4];     /* incoming-wave scheme of each CBC side, Tab. CBCs     */
    int viscous;       /* 0: mesoscopic (Eqs. LaplaceU/T); 1: -FD; 2: none    */
    int dirichlet;     /* 0: equilibrium BC; 1: NEEP (Eq. NEEP); 2: NEEP with the
                          non-equilibrium part regularised (orders 2, 3)       */
    double alpha_T;    /* alpha of Eqs. CBC-Relax / LODI-Relax (transversal)   */
    double beta_P;     /* beta of Eqs. CBC-Relax / LODI-Relax (pressure)       */
    double t_inf;      /* target transversal amplitude T^inf                   */
    double p_inf[4];   /* target pressure Z_inf = P_inf per side (lattice P)   */
    double inflow[4];  /* rho, ux, uy, T imposed on inflow sides               */
    double alpha_V;    /* relaxation of the viscous term towards 0 in Eq.
                          CBC-Relax (an extension; 0 is the paper's equation) */
    int meso_depth;    /* depth below x_f of the first node of the mesoscopic
                          viscous stencil (Sec. 3.3, "Evaluation of viscous
                          terms"); negative: M, the first node none of whose
                          populations was streamed from a boundary layer.  0
                          is x_f itself, the literal reading, kept so a test
                          can show its growth on the Sec. 4.2 vortex.        */
} orc_params;

typedef struct orc_sim orc_sim;

/* Lattice tables (Appendix B).  c has 2*q ints (x,y per velocity). */
int    orc_lattice_info(int lattice, int* q, int* M, double* cs2, int* c, double* w);

/* Shifted equilibrium g_i = f^eq_i - w_i rho0 (Eqs. feq-3/feq-4). */
void   orc_feq(int lattice, double rho0, const double U[4], double* g);
/* Hermite projection of a non-equilibrium vector g[q] onto orders 2 (and 3
 * on the thermal lattices), in place. */
int    orc_regularize(int lattice, double* g);
/* Moments (Eq. macro) of shifted populations: U = (drho, ux, uy, dT). */
void   orc_moments(int lattice, double rho0, const double* g, double U[4]);

/* Characteristic matrices of Sec. 3.1 at a local-frame state
 * Ul = (drho, u_n, u_t, dT).  Thermal: 4x4 row-major; isothermal D2Q9: 3x3
 * stored in the top-left of the 4x4 arrays.  Lam holds the eigenvalues. */
void   orc_char_matrices(int lattice, double rho0, const double Ul[4],
                         double S[16], double Sinv[16], double Lam[4]);

/* Pointwise right-hand side of the boundary ODE (Eqs. thermal_LODI_macro_evo /
 * thermal_CBC_macro_evo with Eqs. PNR, LODI-Relax, CBC-PNR, CBC-Relax) in the
 * local frame, given the normal derivative dUn, the transversal vector TT
 * (script T), the viscous vector VV (script V), the incoming-wave bit mask and
 * the pressure excess dP = P - P_inf. */
void   orc_char_rhs(const orc_params* p, const double Ul[4], const double dUn[4],
                    const double TT[4], const double VV[4], int incoming_mask,
                    double dP, int scheme, double k[4]);

/* Right-hand side of the corner unknown cid (0 SW, 1 SE, 2 NW, 3 NE) from
 * the lab-frame states (drho, ux, uy, dT) of the innermost corner node and
 * of the nodes one and two diagonal steps inward (Sec. 3.3: LODI along the
 * outward diagonal, one-sided difference of spacing sqrt(2)); lab frame. */
int    orc_corner_rhs(const orc_params* p, int cid, const double Uc[4], const double U1[4],
                      const double U2[4], double k[4]);

/* Generic classical RK4 step of size 1 over n unknowns; used by the boundary
 * solver and exported so a test can drive it with a scalar ODE y' = lam y. */
double orc_rk4_scalar(double lam, double y0, double h, int nsteps);

orc_sim* orc_create(const orc_params* p);
void     orc_destroy(orc_sim* s);
/* Initialise f = f^eq(U0) everywhere (Sec. 2, Fig. flowchart-lbm-algo). */
void     orc_init(orc_sim* s, const double* rho, const double* ux,
                  const double* uy, const double* T);
void     orc_step(orc_sim* s, int n);
/* Macroscopic fields (absolute rho, ux, uy, T) of the current populations. */
void     orc_macros(const orc_sim* s, double* rho, double* ux, double* uy, double* T);
/* Shifted populations [ny][nx][q] in the oracle's own velocity order. */
void     orc_populations(const orc_sim* s, double* g);
/* Non-equilibrium moments at node (x,y): sigma'_xx, sigma'_xy, sigma'_yy
 * (Eq. LaplaceU) and q_x, q_y (Eq. LaplaceT, with the (1-1/(2 tau)) factor). */
void     orc_neq_moments(const orc_sim* s, int x, int y, double out[5]);
/* Mesoscopic viscous vector V (local frame of side `side`) with its stencil
 * starting at node (x,y): one-sided normal differences through (x,y),
 * (x,y) - n, (x,y) - 2n and central tangential ones.  The boundary solver
 * evaluates it at x_f - meso_depth n. */
void     orc_vis_meso_at(const orc_sim* s, int side, int x, int y, double V[4]);
/* Boundary state of the last step: U of each node in deviation form,
 * [ny][nx][4]; meaningful on boundary nodes. */
void     orc_boundary_state(const orc_sim* s, double* Ub);
long     orc_steps_done(const orc_sim* s);
int      orc_threads(void);
int      orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
