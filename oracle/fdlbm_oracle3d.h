/* Plain FP64 CPU oracle of the coupled FD-LBM scheme on the D3Q19 lattice.
 *
 * TEST INFRASTRUCTURE ONLY (as fdlbm_oracle.h): the slow reference the CUDA solver's
 * 3D path is checked against. It shares no source, header, table or helper with the
 * CUDA solver library, nor with the D2Q9 oracle.
 *
 * The paper's scheme is stated for D2Q9 and its 3D extension is only announced
 * (Sec. 2). The 3D lattice follows reading R1b: the product-form equilibrium is formed
 * on D3Q27 and each corner population is folded onto its three face diagonals (+), its
 * three axis links (-) and the rest population (+), which keeps the 0th, 1st and 2nd
 * moments (and the third moments c_a c_b^2) of the product form.
 */
#ifndef FDLBM_ORACLE3D_H
#define FDLBM_ORACLE3D_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORA3_MAX_NS 8
#define ORA3_MAX_NR 4
#define ORA3_Q 19

/* Problem description, every array host-owned and copied at ora3_create. */
typedef struct {
  int nx, ny, nz;                  /* D3Q19 lattice size */
  const unsigned char* mask;       /* nx*ny*nz, x fastest then y: 0 gas, 1 inert, 2 catalytic */
  int face_bc[6];                  /* x-, x+, y-, y+, z-, z+: 0 periodic 1 inlet 2 outlet 3 closed 4 fixed-T */
  int ns;
  double M_gmol[ORA3_MAX_NS];
  double tau1[ORA3_MAX_NS], tau2[ORA3_MAX_NS];
  double X_init[ORA3_MAX_NS], X_inlet[ORA3_MAX_NS];
  double Pr; int energy_correction;
  double T0_K, T_init_K, T_inlet_K, T_solid_init_K, T_outer_K;
  double u_inlet;                  /* plug inlet along +x */
  double alpha_s, rhocp_s, kappa_f; int coupling; /* 0 conservative, 1 paper law */
  int nr;
  int nu[ORA3_MAX_NR][ORA3_MAX_NS];
  double k0[ORA3_MAX_NR], Ea_Jmol[ORA3_MAX_NR], Keq[ORA3_MAX_NR], dH_Jmol[ORA3_MAX_NR];
  int rate_form[ORA3_MAX_NR];
  double rho_w_tol; int rho_w_maxit;
  const double* init_X;   /* optional [ns][n] */
  const double* init_u;   /* optional [3][n] */
  const double* init_T;   /* optional [n], K */
  const double* init_Ts;  /* optional [n], K */
  const double* init_C;   /* optional [n], lattice molar concentration (default 1) */
  /* Time level of the energy-correction gradients (reading R8): 0, the moments of this
   * step; 1, those of the previous step. */
  int phi_lagged;
} ora3_problem;

typedef struct ora3_state ora3_state;

/* Ledger layout of ora3_balance: the same as the D2Q9 oracle's. */
enum {
  ORA3_B_STEPS = 0, ORA3_B_E_GAS, ORA3_B_E_GAS0, ORA3_B_H_SOLID, ORA3_B_H_SOLID0,
  ORA3_B_Q_RXN, ORA3_B_Q_WALL, ORA3_B_Q_COUPLE, ORA3_B_Q_FIXEDT, ORA3_B_RESIDUAL,
  ORA3_B_SOLID_RESIDUAL, ORA3_B_EPS_PAPER, ORA3_B_NOCONV, ORA3_B_MASS
};

/* Exact accounts of ora3_accounts: the layout of the D2Q9 oracle's ORA_A_*. */
enum {
  ORA3_A_E_POP = 0, ORA3_A_E_POP0, ORA3_A_Q_INLET, ORA3_A_Q_OUTLET, ORA3_A_D_INTERP, ORA3_A_D_COLLISION,
  ORA3_A_D_COUPLING, ORA3_A_CLOSURE, ORA3_A_MASS /* then 8 blocks of ns */
};

ora3_state* ora3_create(const ora3_problem* p, char* err, int errlen);
void ora3_destroy(ora3_state* s);
int ora3_step(ora3_state* s, int nsteps);
int ora3_nfields(const ora3_state* s);                 /* 2*ns + 5 */
void ora3_moments(const ora3_state* s, double* out);   /* rho_j, X_j, ux, uy, uz, T_K (gas), Ts_K (solid) */
void ora3_populations(const ora3_state* s, double* out); /* [ns][19][n] */
/* State the next step reads (g [ns][19][n], T_s [n], gas T [n], lattice units); the
 * slab decomposition's exchange reads and overwrites its ghost strips through these. */
void ora3_get_state(const ora3_state* s, double* g, double* Ts, double* T);
void ora3_set_state(ora3_state* s, const double* g, const double* Ts, const double* T);
void ora3_balance(const ora3_state* s, double* out);
/* Exact accounts (energy, then per-species mass; layout ORA3_A_*). */
void ora3_accounts(const ora3_state* s, double* out);
double ora3_residual(ora3_state* s, int K);
void ora3_counts(const ora3_state* s, long* out);      /* class counts [5] + stencil counts [6] */
void ora3_classes(const ora3_state* s, int* out);

/* Point functions for the pins. Velocity set: index i has components
 * ora3_velocity(i, out3) (rest, 6 axis links, 12 face diagonals). */
void ora3_velocity(int i, int* out3);
/* One link's interpolated pull (the 3D oracle's own copy of the Sec. 4.2 stencils): code
 * as for the D2Q9 oracle (0 none, 1 central, 2 forward, 3 backward, 4/5 linear). */
double ora3_interp(int code, double c, double s3, double s2, double s1, double s0, double sp);
void ora3_equilibrium(double rho, double ux, double uy, double uz, double M, double T, double* f19);
void ora3_psi(double c, double* px, double* py, double* pz);
void ora3_phi(double c, double* phi);
void ora3_collide(int ns, const double* M, const double* tau1, const double* tau2,
                  const double* g /* [ns][19] */, const double* divq /* [ns] */,
                  double* gout /* [ns][19] */, double* mom /* rho_j[ns], ux, uy, uz, T, Tg */);

#ifdef __cplusplus
}
#endif
#endif
