/* Plain FP64 CPU oracle of the coupled finite-difference / lattice-Boltzmann scheme
 * for catalytic flow (Kulyk, Berger, Smith, Harting, arXiv:1804.07588).
 *
 * TEST INFRASTRUCTURE ONLY. This is the slow, obviously-correct reference that the
 * CUDA solver is checked against. Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg load it. It shares no source, header, table or helper
 * with the CUDA solver library.
 *
 * Scope: D2Q9 lattice (the paper's lattice, Sec. 2, Eq. cx).
 */
#ifndef FDLBM_ORACLE_H
#define FDLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORA_MAX_NS 8
#define ORA_MAX_NR 4

/* Problem description, every array host-owned and copied at ora_create. */
typedef struct {
  int nx, ny;                      /* D2Q9 lattice size */
  const unsigned char* mask;       /* nx*ny, x fastest: 0 gas, 1 inert solid, 2 catalytic */
  int face_bc[4];                  /* x-, x+, y-, y+: 0 periodic 1 inlet 2 outlet 3 closed 4 fixed-T */
  int ns;                          /* species count */
  double M_gmol[ORA_MAX_NS];       /* molar masses (scaled by the lightest inside) */
  double tau1[ORA_MAX_NS], tau2[ORA_MAX_NS];
  double X_init[ORA_MAX_NS], X_inlet[ORA_MAX_NS];
  double Pr; int energy_correction;
  double T0_K, T_init_K, T_inlet_K, T_solid_init_K, T_outer_K;
  double u_inlet; int inlet_profile;          /* 0 plug, 1 parabolic */
  double alpha_s, rhocp_s, kappa_f; int coupling; /* 0 conservative, 1 paper law */
  int nr;
  int nu[ORA_MAX_NR][ORA_MAX_NS];
  double k0[ORA_MAX_NR], Ea_Jmol[ORA_MAX_NR], Keq[ORA_MAX_NR], dH_Jmol[ORA_MAX_NR];
  int rate_form[ORA_MAX_NR];                  /* 0 concentration bilinear, 1 mole-fraction reversible */
  double rho_w_tol; int rho_w_maxit;
  const double* init_X;   /* optional [ns][n] mole fractions */
  const double* init_u;   /* optional [2][n] */
  const double* init_T;   /* optional [n] gas temperature, K */
  const double* init_Ts;  /* optional [n] solid temperature, K */
  const double* init_C;   /* optional [n] molar concentration (lattice, default 1) */
  /* Locally updated relaxation times (local_tau = 1): per node, tau1_j from the species
   * viscosities mu_j by Wilke's mixture rule (Eq. tau1s) and tau2_j from the binary
   * diffusivities D_jk by the mixture-averaged rule (Eqs. tau2_approx_text, D_j_text);
   * tau1/tau2 above are then unused. Lattice units. */
  int local_tau;
  double mu[ORA_MAX_NS];
  double Djk[ORA_MAX_NS][ORA_MAX_NS];
  /* Optional [2][n] velocity of solid nodes (lattice): a moving diffusive wall emits
   * f^eq(1, U_w, T_w) (Eq. BC_g_ji_1 with the wall velocity); NULL: walls at rest. */
  const double* wall_u;
  /* Time level of the energy-correction gradients (reading R8): 0, the moments of this
   * step (the plain reading of Eq. final_kinetic_equation); 1, those of the previous
   * step. */
  int phi_lagged;
} ora_problem;

typedef struct ora_state ora_state;

/* Ledger layout returned by ora_balance (all lattice energy units). */
enum {
  ORA_B_STEPS = 0, ORA_B_E_GAS, ORA_B_E_GAS0, ORA_B_H_SOLID, ORA_B_H_SOLID0,
  ORA_B_Q_RXN, ORA_B_Q_WALL, ORA_B_Q_COUPLE, ORA_B_Q_FIXEDT, ORA_B_RESIDUAL, ORA_B_SOLID_RESIDUAL,
  ORA_B_EPS_PAPER, ORA_B_NOCONV, ORA_B_MASS /* then mass[ns], mass0[ns], moles[ns], moles0[ns] */
};

/* Exact accounts returned by ora_accounts: the inventory of the stored populations (gas
 * post-collision populations and wall emissions in transit) now and at the start, the
 * shift-sense inlet and outlet fluxes, the interpolation, collision and coupling
 * defects and the energy closure; then per species (ns each) the mass inventory now
 * and at the start, inlet and outlet mass fluxes, interpolation and collision mass
 * defects, reaction production at the walls and the mass closure. */
enum {
  ORA_A_E_POP = 0, ORA_A_E_POP0, ORA_A_Q_INLET, ORA_A_Q_OUTLET, ORA_A_D_INTERP, ORA_A_D_COLLISION,
  ORA_A_D_COUPLING, ORA_A_CLOSURE, ORA_A_MASS /* then 8 blocks of ns */
};

ora_state* ora_create(const ora_problem* p, char* err, int errlen);
void ora_destroy(ora_state* s);
int ora_step(ora_state* s, int nsteps);
int ora_nfields(const ora_state* s);                 /* 2*ns + 4 */
void ora_moments(const ora_state* s, double* out);   /* [field][n]: rho_j, X_j, ux, uy, T_K, Ts_K */
void ora_populations(const ora_state* s, double* out); /* [ns][9][n] stored post-collision / wall-emitted */
/* The state a step reads: populations g [ns][9][n], solid temperature Ts [n] and gas
 * temperature T [n] (lattice units); NULL arrays are skipped. Used to exchange the ghost
 * columns of slabs that each run their own oracle (the slab decomposition's check). */
void ora_get_state(const ora_state* s, double* g, double* Ts, double* T);
void ora_set_state(ora_state* s, const double* g, const double* Ts, const double* T);
void ora_balance(const ora_state* s, double* out);
/* Exact accounts (energy, then per-species mass; layout ORA_A_*). */
void ora_accounts(const ora_state* s, double* out);
double ora_residual(ora_state* s, int K);
void ora_counts(const ora_state* s, long* out);      /* class counts [5] + stencil counts [6] */
void ora_classes(const ora_state* s, int* out);      /* per-node class */

/* Point functions exposed so that the test-suite can pin them individually. */
void ora_units(double T0_K, double M0_gmol, double dx_m, double* out3);
void ora_equilibrium(double rho, double ux, double uy, double M, double T, double* f9);
double ora_interp(int code, double c, double s3, double s2, double s1, double s0, double sp);
void ora_psi(double c, double* psix9, double* psiy9);
void ora_phi(double c, double* phi9);
double ora_uc(int ns, const double* rho, const double* Jx, const double* tau2, double ux);
/* Wilke's coefficient phi_jk (Eq. wilke, read with the squared bracket). */
double ora_wilke_phi(double mu_j, double mu_k, double M_j, double M_k);
/* Local relaxation times of one node from its species densities rho[ns], molar masses
 * M[ns] and temperature T (Eqs. tau1s, tau2_approx_text, D_j_text). */
void ora_local_tau(int ns, const double* M, const double* mu, const double* Djk /* [ns][ORA_MAX_NS] */,
                   const double* rho, double T, double* tau1, double* tau2);
void ora_collide(int ns, const double* M, const double* tau1, const double* tau2,
                 const double* g /* [ns][9] pulled */, const double* divq /* [ns] */,
                 double* gout /* [ns][9] */, double* mom /* rho_j[ns], ux, uy, T, Tg */);

#ifdef __cplusplus
}
#endif
#endif
