/* Plain FP64 CPU oracle of the coupled FD-LBM scheme for catalytic flow
 * (Kulyk, Berger, Smith, Harting, arXiv:1804.07588).
 *
 * TEST INFRASTRUCTURE ONLY: the slow reference the CUDA solver is checked against.
 * It is deliberately written as plain loops over lattice nodes, one pass per step of
 * the algorithm, in the order the paper's equations are stated. It shares no code with
 * the CUDA solver. Where the paper is silent or garbled, the reading taken is stated at
 * the point of use (tagged R1..R16; the same tags index the list of readings kept with
 * the project's design notes).
 *
 * One time step t -> t+1 (reading R14; the paper does not fix the order). Every pass
 * reads time level t only:
 *   1. wall pass: at every gas-solid interface (wall) node, the populations arriving
 *      from the gas are streamed in from g*(t), the wall density is iterated with the
 *      surface reaction (Sec. 4.3, Eqs. mass_balance, BC_g_ji_1, BC_gji) and the wall
 *      emits its unknown populations w(t+1); reaction heat and the energy the wall puts
 *      into the gas are recorded per wall node;
 *   2. solid pass: explicit FD heat step on solid nodes (Eqs. heat_equation_fd,
 *      heat_equation_fd_2nd_deriv) with the interface coupling (Eq. wall_temperature or
 *      its conservative reading R12) and the reaction heat, plus the ledger fluxes;
 *   3. gas pass: every gas node pulls g*(t) (wall emissions w(t) included) with the
 *      off-lattice quadratic interpolation (Sec. 4.2), takes its moments (Eq.
 *      moments_of_g), the energy-correction divergence on its 4 axis neighbours (from
 *      the moments of this step, reading R8; optionally those of the previous time
 *      level) and collides (Eq. final_kinetic_equation).
 */
#include "fdlbm_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define Q 9
/* D2Q9 velocities of the lightest species, Eq. cx. */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

static const double R_GAS = 8.314462618; /* J/(mol K) */

enum { CL_GAS = 0, CL_INLET = 1, CL_OUTLET = 2, CL_WALL = 3, CL_SOLID = 4 };
enum { F_PERIODIC = 0, F_INLET = 1, F_OUTLET = 2, F_CLOSED = 3, F_FIXED_T = 4 };
enum { ST_NONE = 0, ST_CENTRAL = 1, ST_FORWARD = 2, ST_BACKWARD = 3, ST_LIN_S0 = 4, ST_LIN_S2 = 5 };

struct ora_state {
  ora_problem p;
  int nx, ny, n, ns;
  unsigned char* mask;
  int* cls;
  double M[ORA_MAX_NS], c[ORA_MAX_NS];
  double T0;                 /* reference temperature, K: lattice T = T_K / (3 T0) */
  double* g;                 /* [ns][Q][n] post-collision (gas, inlet, outlet) and wall emissions */
  double* gn;
  double* gp;                /* [ns][Q][n] pulled (pre-collision) populations of gas nodes */
  double* Ts;                /* [n] solid temperature, lattice units */
  double* Tsn;
  double* rho;               /* [ns][n] f-moments at the current time (gas nodes) */
  double* ux;
  double* uy;
  double* T;                 /* mixture temperature T(f), lattice units */
  double* Tg;                /* g-temperature of the current step */
  double* Cj;                /* [ns][n] concentrations of the current step */
  double* Tg_prev;           /* g-temperature of the previous time level (reading R8) */
  double* Cj_prev;           /* [ns][n] concentrations of the previous time level */
  double* divq;              /* scratch [ns][n] */
  double* tau1_prev;         /* [ns][n] local tau1 of the previous time level (local_tau) */
  double* tau1_cur;          /* [ns][n] tau1 of every gas node at this step */
  double* tau2_cur;          /* [ns][n] tau2 of every gas node at this step */
  double* wall_u;            /* [2][n] wall velocity of solid nodes */
  double* q;                 /* [n] reaction heat of the step at wall nodes */
  double* dE;                /* [n] energy the wall put into the gas this step */
  double* snap;              /* residual snapshot */
  int have_snap;
  double steps;
  double E_gas0, H_solid0, mass0[ORA_MAX_NS], moles0[ORA_MAX_NS];
  double Q_rxn, Q_wall, Q_couple, Q_fixedT, noconv;
  /* Exact accounts (ora_accounts): inventory of the stored populations at the start,
   * shift-sense inlet/outlet fluxes, interpolation and collision defects (energy and
   * per-species mass) and the mass the reactions produce at the walls. */
  double E_pop0, Q_in, Q_out, D_int, D_col;
  double Mpop0[ORA_MAX_NS], M_in[ORA_MAX_NS], M_out[ORA_MAX_NS], Dm_int[ORA_MAX_NS], Dm_col[ORA_MAX_NS],
      M_rxn[ORA_MAX_NS];
  long st_count[6];
};

/* ------------------------------------------------------------------------------------
 * Lattice helpers
 * ---------------------------------------------------------------------------------- */
static int periodic_x(const ora_state* s) { return s->p.face_bc[0] == F_PERIODIC; }
static int periodic_y(const ora_state* s) { return s->p.face_bc[2] == F_PERIODIC; }

/* Node index of (x, y), wrapped on periodic axes; -1 outside the lattice. */
static int node_at(const ora_state* s, int x, int y) {
  if (x < 0 || x >= s->nx) {
    if (!periodic_x(s)) return -1;
    x = ((x % s->nx) + s->nx) % s->nx;
  }
  if (y < 0 || y >= s->ny) {
    if (!periodic_y(s)) return -1;
    y = ((y % s->ny) + s->ny) % s->ny;
  }
  return x + s->nx * y;
}

static int cls_at(const ora_state* s, int x, int y) {
  int k = node_at(s, x, y);
  return k < 0 ? -1 : s->cls[k];
}

static size_t PIDX(const ora_state* s, int j, int i, int k) {
  return ((size_t)j * Q + (size_t)i) * (size_t)s->n + (size_t)k;
}

/* Does node (x, y) hold a post-collision population moving in direction i?  Gas,
 * inlet and outlet nodes emit every direction; a wall node emits direction i only
 * towards a gas neighbour (the unknown populations of Eq. BC_gji). Reading R6. */
static int source_exists(const ora_state* s, int x, int y, int i) {
  int c = cls_at(s, x, y);
  if (c == CL_GAS || c == CL_INLET || c == CL_OUTLET) return 1;
  if (c == CL_WALL) return cls_at(s, x + EX[i], y + EY[i]) == CL_GAS;
  return 0;
}

/* Stencil choice for pulling direction i into target (x, y) (reading R6): the paper's
 * central form where both neighbouring off-lattice points exist (Eq. interpol_bulk),
 * the forward form where the upstream one is missing (Eq. interpol_away), the backward
 * form where the downstream one is missing (Eq. interpol_towards), and linear or no
 * interpolation where even those lack a point (concave corners and one-node gaps,
 * which the paper excludes from its geometries). */
static int stencil_code(const ora_state* s, int x, int y, int i) {
  int e2 = source_exists(s, x - 2 * EX[i], y - 2 * EY[i], i);
  int e0 = source_exists(s, x, y, i);
  int ep = source_exists(s, x + EX[i], y + EY[i], i);
  int e3 = source_exists(s, x - 3 * EX[i], y - 3 * EY[i], i);
  if (e2 && e0) return ST_CENTRAL;
  if (e0 && ep) return ST_FORWARD;
  if (e2 && e3) return ST_BACKWARD;
  if (e0) return ST_LIN_S0;
  if (e2) return ST_LIN_S2;
  return ST_NONE;
}

/* Quadratic upwind interpolation of Sec. 4.2 (Eq. interpol_general): the on-lattice
 * value is the off-lattice value s1 (streamed from x - e_i) advanced by (1 - c) with
 * first and second differences of neighbouring off-lattice values. s2, s3 are streamed
 * from x - 2e_i, x - 3e_i, s0 from x itself and sp from x + e_i. */
double ora_interp(int code, double c, double s3, double s2, double s1, double s0, double sp) {
  double a = 1.0 - c;
  double d1, d2;
  switch (code) {
    case ST_CENTRAL: /* Eq. interpol_bulk */
      d1 = (s0 - s2) / 2.0;
      d2 = s0 - 2.0 * s1 + s2;
      break;
    case ST_FORWARD: /* Eq. interpol_away: B = s1, C = s0, D = sp */
      d1 = (4.0 * s0 - sp - 3.0 * s1) / 2.0;
      d2 = -2.0 * s0 + sp + s1;
      break;
    case ST_BACKWARD: /* Eq. interpol_towards: Z = s1, Y = s2, X = s3 */
      d1 = -(4.0 * s2 - s3 - 3.0 * s1) / 2.0;
      d2 = -2.0 * s2 + s3 + s1;
      break;
    case ST_LIN_S0:
      return s1 + a * (s0 - s1);
    case ST_LIN_S2:
      return s1 + a * (s1 - s2);
    default:
      return s1;
  }
  return s1 + d1 * a + d2 * 0.5 * a * a;
}

/* Value of population (j, i) pulled into target (x, y) from the array gsrc. */
static double pull(ora_state* s, const double* gsrc, int j, int i, int x, int y, int count) {
  int k0 = node_at(s, x, y);
  if (i == 0) return gsrc[PIDX(s, j, 0, k0)];
  int code = stencil_code(s, x, y, i);
  if (count) s->st_count[code]++;
  int k1 = node_at(s, x - EX[i], y - EY[i]);
  double s1 = gsrc[PIDX(s, j, i, k1)];
  double s0 = 0, s2 = 0, s3 = 0, sp = 0;
  if (code == ST_CENTRAL || code == ST_FORWARD || code == ST_LIN_S0) s0 = gsrc[PIDX(s, j, i, k0)];
  if (code == ST_CENTRAL || code == ST_BACKWARD || code == ST_LIN_S2)
    s2 = gsrc[PIDX(s, j, i, node_at(s, x - 2 * EX[i], y - 2 * EY[i]))];
  if (code == ST_BACKWARD) s3 = gsrc[PIDX(s, j, i, node_at(s, x - 3 * EX[i], y - 3 * EY[i]))];
  if (code == ST_FORWARD) sp = gsrc[PIDX(s, j, i, node_at(s, x + EX[i], y + EY[i]))];
  return ora_interp(code, s->c[j], s3, s2, s1, s0, sp);
}

/* The pure-shift value of a pull: population (j, i) of the node x - e_i (the node
 * itself for the rest population). */
static double shift_source(const ora_state* s, const double* gsrc, int j, int i, int x, int y) {
  return gsrc[PIDX(s, j, i, node_at(s, x - EX[i], y - EY[i]))];
}

/* Energy weight of population (j, i): (1/2) c_j^2 |e_i|^2. */
static double eps_w(const ora_state* s, int j, int i) {
  return 0.5 * s->c[j] * s->c[j] * (double)(EX[i] * EX[i] + EY[i] * EY[i]);
}

/* ------------------------------------------------------------------------------------
 * Equilibria, correction coefficients, collision
 * ---------------------------------------------------------------------------------- */

/* One Cartesian factor of the product-form equilibrium, Eq. eq_state_pop (reading R1:
 * the printed prefactor (1 - 2c^2) / 2^(c^2) flips the sign of every factor, and the two
 * flips cancel in the D2Q9 product; the factor is written here with the sign that makes
 * it positive). e is the lattice component (-1, 0, 1), v the velocity component. */
static double wfac(int e, double v, double M, double T) {
  if (e == 0) return 1.0 - M * v * v - T;
  return 0.5 * ((double)e * sqrt(M) * v + M * v * v + T);
}

/* f^eq_i(rho, u, T) of species mass M (Eq. eq_state_pop); with the species velocity in
 * place of u it is the auxiliary quasi-equilibrium f* (Eq. aux_state_pop). */
void ora_equilibrium(double rho, double ux, double uy, double M, double T, double* f9) {
  for (int i = 0; i < Q; ++i) f9[i] = rho * wfac(EX[i], ux, M, T) * wfac(EY[i], uy, M, T);
}

/* Forcing coefficients psi_ji (Eq. psi_jialpha). */
void ora_psi(double c, double* px, double* py) {
  static const double PX[Q] = {0, 4, 0, -4, 0, -1, 1, 1, -1};
  static const double PY[Q] = {0, 0, 4, 0, -4, -1, -1, 1, 1};
  for (int i = 0; i < Q; ++i) {
    px[i] = PX[i] / (4.0 * c);
    py[i] = PY[i] / (4.0 * c);
  }
}

/* Energy-only coefficients phi_ji of the Prandtl correction (Eq. forcing_correction_Pr).
 * The paper does not print them (reading R4): -1 at rest, 1/(2D) on the axis links, 0 on
 * diagonals, over c_j^2. This has zero mass and momentum and unit energy moment. */
void ora_phi(double c, double* phi) {
  for (int i = 0; i < Q; ++i) phi[i] = 0.0;
  phi[0] = -1.0 / (c * c);
  for (int i = 1; i <= 4; ++i) phi[i] = 0.25 / (c * c);
}

/* Corrective diffusion velocity U^c (Eq. correction_diffusion_velocities_final, reading
 * R3): the trapezoidal (g-form) collision conserves the mixture momentum exactly when
 * the weights 1/tau_j2 of the continuous formula become 1/(tau_j2 + 1/2) with the g
 * moments J_j(g), u = J(g)/rho. One Cartesian component. */
double ora_uc(int ns, const double* rho, const double* Jx, const double* tau2, double ux) {
  double num = 0.0, den = 0.0;
  for (int j = 0; j < ns; ++j) {
    num += (Jx[j] - rho[j] * ux) / (tau2[j] + 0.5);
    den += rho[j] / (tau2[j] + 0.5);
  }
  return num / den;
}

/* Wilke's mixture rule (Eq. wilke). The printed coefficient lacks the square on the
 * bracket; without it a pure gas (phi_jj = 2 / 4) would have twice its own viscosity, so
 * the bracket is squared as in Wilke's rule (phi_jj = 1). */
double ora_wilke_phi(double mu_j, double mu_k, double M_j, double M_k) {
  double b = 1.0 + sqrt(mu_j / mu_k) * pow(M_k / M_j, 0.25);
  return b * b / sqrt(8.0 * (1.0 + M_j / M_k));
}

/* Locally updated relaxation times of one node (Sec. 3): tau1_j = mu_j / (C T sum_k X_k
 * phi_jk) (Eq. tau1s), tau2_j = rho_j D_j / (X_j p) with p = C T (Eq. tau2_approx_text)
 * and the mixture-averaged D_j = (1 - Y_j) / sum_{k != j} X_k / D_jk (Eq. D_j_text).
 * X_j mole fractions, Y_j mass fractions. For an empty species (X_j = 0) rho_j / X_j is
 * replaced by its limit M_j C. */
void ora_local_tau(int ns, const double* M, const double* mu, const double* Djk, const double* rho, double T,
                   double* tau1, double* tau2) {
  double C = 0.0, r = 0.0, X[ORA_MAX_NS];
  for (int j = 0; j < ns; ++j) {
    C += rho[j] / M[j];
    r += rho[j];
  }
  for (int j = 0; j < ns; ++j) X[j] = rho[j] / M[j] / C;
  double p = C * T;
  for (int j = 0; j < ns; ++j) {
    double s = 0.0;
    for (int k = 0; k < ns; ++k) s += X[k] * ora_wilke_phi(mu[j], mu[k], M[j], M[k]);
    tau1[j] = mu[j] / (C * T * s);
    double sd = 0.0;
    for (int k = 0; k < ns; ++k)
      if (k != j) sd += X[k] / Djk[j * ORA_MAX_NS + k];
    double Dj = (1.0 - rho[j] / r) / sd;
    double rho_over_X = X[j] > 0.0 ? rho[j] / X[j] : M[j] * C;
    tau2[j] = rho_over_X * Dj / p;
  }
}

/* Moments of pulled g of one node (Eq. moments_of_g, first line, and Eq. moments_of_f). */
static void g_moments(int ns, const double* M, const double* g, double* rho, double* Jx,
                      double* Jy, double* E) {
  for (int j = 0; j < ns; ++j) {
    double c = 1.0 / sqrt(M[j]);
    double r = 0, jx = 0, jy = 0, e = 0;
    for (int i = 0; i < Q; ++i) {
      double v = g[j * Q + i];
      r += v;
      jx += c * EX[i] * v;
      jy += c * EY[i] * v;
      e += c * c * (EX[i] * EX[i] + EY[i] * EY[i]) * v;
    }
    rho[j] = r;
    Jx[j] = jx;
    Jy[j] = jy;
    E[j] = e;
  }
}

/* g-temperature (E(g) - J(g)^2/rho) / (2C) (first part of Eq. moments_of_g, third line). */
static double g_temperature(int ns, const double* M, const double* g, double* Cj_out) {
  double rho[ORA_MAX_NS], Jx[ORA_MAX_NS], Jy[ORA_MAX_NS], E[ORA_MAX_NS];
  g_moments(ns, M, g, rho, Jx, Jy, E);
  double r = 0, jx = 0, jy = 0, e = 0, C = 0;
  for (int j = 0; j < ns; ++j) {
    r += rho[j];
    jx += Jx[j];
    jy += Jy[j];
    e += E[j];
    C += rho[j] / M[j];
    if (Cj_out) Cj_out[j] = rho[j] / M[j];
  }
  return (e - (jx * jx + jy * jy) / r) / (2.0 * C);
}

/* Collision of one gas node, Eq. final_kinetic_equation with dt = 1:
 *   g' = g - w1 (g - f*) - w1 (tau1/tau2)(f* - f^eq) + w1 tau1 (Psi + Phi),
 *   w1 = 2 / (1 + 2 tau1),
 * with the f-moments taken from g by Eq. moments_of_g: J_j(f) from J_j(g), the
 * equilibrium momentum rho_j u and the Psi momentum rho_j U^c / tau2; T(f) from the g
 * temperature plus the Phi energy term sum_ji c^2 Phi_ji / (4C) = sum_j divq_j / (4C).
 * divq_j is the divergence of the Prandtl heat flux q^Pr_j (Eq. q_Pr) at this node. */
void ora_collide(int ns, const double* M, const double* tau1, const double* tau2,
                 const double* g, const double* divq, double* gout, double* mom) {
  double rho[ORA_MAX_NS], Jx[ORA_MAX_NS], Jy[ORA_MAX_NS], E[ORA_MAX_NS];
  g_moments(ns, M, g, rho, Jx, Jy, E);
  double r = 0, jx = 0, jy = 0, e = 0, C = 0, sdq = 0;
  for (int j = 0; j < ns; ++j) {
    r += rho[j];
    jx += Jx[j];
    jy += Jy[j];
    e += E[j];
    C += rho[j] / M[j];
    sdq += divq[j];
  }
  double ux = jx / r, uy = jy / r;
  double Tg = (e - (jx * jx + jy * jy) / r) / (2.0 * C);
  double T = Tg + sdq / (4.0 * C);
  double Ucx = ora_uc(ns, rho, Jx, tau2, ux);
  double Ucy = ora_uc(ns, rho, Jy, tau2, uy);
  for (int j = 0; j < ns; ++j) {
    double c = 1.0 / sqrt(M[j]);
    double a = 1.0 / (2.0 * tau2[j]);
    double Jfx = (Jx[j] + a * rho[j] * (ux + Ucx)) / (1.0 + a);
    double Jfy = (Jy[j] + a * rho[j] * (uy + Ucy)) / (1.0 + a);
    /* Species velocity of f* (Eq. aux_state_pop). Reading R15: an empty species takes the
     * mixture velocity, and each component is limited to |u| <= sqrt((1 - T) / M_j), the
     * range where the rest factor of the product-form equilibrium stays non-negative;
     * the limit only acts on trace species whose density the interpolation has driven
     * to (or through) zero, and keeps f* -> 0 continuously as rho_j -> 0. */
    double ujx = ux, ujy = uy;
    if (rho[j] != 0.0) {
      double lim = sqrt((1.0 - T) / M[j]);
      ujx = Jfx / rho[j];
      ujy = Jfy / rho[j];
      ujx = ujx > lim ? lim : (ujx < -lim ? -lim : ujx);
      ujy = ujy > lim ? lim : (ujy < -lim ? -lim : ujy);
    }
    double feq[Q], fst[Q], px[Q], py[Q], phi[Q];
    ora_equilibrium(rho[j], ux, uy, M[j], T, feq);
    ora_equilibrium(rho[j], ujx, ujy, M[j], T, fst);
    ora_psi(c, px, py);
    ora_phi(c, phi);
    double w1 = 2.0 / (1.0 + 2.0 * tau1[j]);
    for (int i = 0; i < Q; ++i) {
      double Psi = (px[i] * Ucx + py[i] * Ucy) * rho[j] / tau2[j]; /* Eq. forcing_correction_diffusion_velocities */
      double Phi = phi[i] * divq[j];                                /* Eq. forcing_correction_Pr */
      double gi = g[j * Q + i];
      gout[j * Q + i] = gi - w1 * (gi - fst[i]) - w1 * (tau1[j] / tau2[j]) * (fst[i] - feq[i]) +
                        w1 * tau1[j] * (Psi + Phi);
    }
  }
  if (mom) {
    for (int j = 0; j < ns; ++j) mom[j] = rho[j];
    mom[ns] = ux;
    mom[ns + 1] = uy;
    mom[ns + 2] = T;
    mom[ns + 3] = Tg;
  }
}

/* ------------------------------------------------------------------------------------
 * Surface kinetics (Eq. showcase_Sj and the reversible mole-fraction law, reading R11)
 * ---------------------------------------------------------------------------------- */

/* Reaction rates (lattice moles per wall node per step) at wall densities rho_w. */
static void rates(const ora_state* s, const double* rho_w, double Tw, double* rate) {
  int ns = s->ns;
  double Cw[ORA_MAX_NS], Ct = 0;
  for (int j = 0; j < ns; ++j) {
    Cw[j] = rho_w[j] / s->M[j];
    Ct += Cw[j];
  }
  double TK = 3.0 * s->T0 * Tw;
  for (int r = 0; r < s->p.nr; ++r) {
    double k = s->p.k0[r] * exp(-s->p.Ea_Jmol[r] / (R_GAS * TK));
    if (s->p.rate_form[r] == 0) {
      double prod = 1.0;
      for (int j = 0; j < ns; ++j)
        for (int m = 0; m < -s->p.nu[r][j]; ++m) prod *= Cw[j];
      rate[r] = k * prod;
    } else {
      double fwd = 1.0, bwd = 1.0;
      for (int j = 0; j < ns; ++j) {
        double xj = Cw[j] / Ct;
        for (int m = 0; m < -s->p.nu[r][j]; ++m) fwd *= xj;
        for (int m = 0; m < s->p.nu[r][j]; ++m) bwd *= xj;
      }
      rate[r] = k * (fwd - bwd / s->p.Keq[r]);
    }
  }
}

/* Rest-equilibrium weight of direction i at temperature T (f^eq(1, 0, T), Eq.
 * BC_g_ji_1 with U_w = 0). It does not depend on the species mass. */
static double wrest(int i, double T) { return wfac(EX[i], 0.0, 1.0, T) * wfac(EY[i], 0.0, 1.0, T); }

/* Unit system of Sec. 4.1: the lightest species moves one lattice spacing per step at
 * the characteristic speed U' = sqrt(3 R T0 / M0), so dt = dx / U'; the lattice
 * temperature unit is T0 / (1/3). out = {U' (m/s), dt (s), kelvin per lattice unit}. */
void ora_units(double T0_K, double M0_gmol, double dx_m, double* out) {
  double U = sqrt(3.0 * R_GAS * T0_K / (M0_gmol * 1e-3));
  out[0] = U;
  out[1] = dx_m / U;
  out[2] = 3.0 * T0_K;
}

/* ------------------------------------------------------------------------------------
 * Set-up
 * ---------------------------------------------------------------------------------- */
static void* xcalloc(size_t n, size_t sz) {
  void* p = calloc(n ? n : 1, sz);
  if (!p) {
    fprintf(stderr, "oracle: out of memory\n");
    abort();
  }
  return p;
}

static int fail(char* err, int errlen, const char* msg, int x, int y) {
  if (err && errlen > 0) snprintf(err, (size_t)errlen, "%s at (%d,%d)", msg, x, y);
  return -1;
}

/* Inlet velocity at inlet node (0, y): plug, or a parabola vanishing on the wall nodes
 * that bound the contiguous inlet run (reading R13; the wall sits on the solid node). */
static double inlet_u(const ora_state* s, int y) {
  if (s->p.inlet_profile == 0) return s->p.u_inlet;
  int y0 = y, y1 = y;
  while (y0 - 1 >= 0 && s->cls[0 + s->nx * (y0 - 1)] == CL_INLET) --y0;
  while (y1 + 1 < s->ny && s->cls[0 + s->nx * (y1 + 1)] == CL_INLET) ++y1;
  double H = (double)(y1 - y0 + 2);
  double sy = (double)(y - y0 + 1) / H;
  return 4.0 * s->p.u_inlet * sy * (1.0 - sy);
}

static void fill_moments_from_fields(ora_state* s, int k, const double* X, double ux, double uy,
                                     double T) {
  for (int j = 0; j < s->ns; ++j) s->rho[(size_t)j * s->n + k] = X[j] * s->M[j];
  s->ux[k] = ux;
  s->uy[k] = uy;
  s->T[k] = T;
}

static void ledger_totals(const ora_state* s, double* E, double* H, double* mass, double* moles);
static void pop_totals(const ora_state* s, double* E, double* mass);

ora_state* ora_create(const ora_problem* p, char* err, int errlen) {
  if (p->nx < 1 || p->ny < 1 || p->ns < 1 || p->ns > ORA_MAX_NS || p->nr < 0 || p->nr > ORA_MAX_NR) {
    fail(err, errlen, "bad sizes", p->nx, p->ny);
    return NULL;
  }
  if ((p->face_bc[0] == F_PERIODIC) != (p->face_bc[1] == F_PERIODIC) ||
      (p->face_bc[2] == F_PERIODIC) != (p->face_bc[3] == F_PERIODIC) ||
      p->face_bc[1] == F_INLET || p->face_bc[0] == F_OUTLET || p->face_bc[2] == F_INLET ||
      p->face_bc[2] == F_OUTLET || p->face_bc[3] == F_INLET || p->face_bc[3] == F_OUTLET) {
    fail(err, errlen, "unsupported face boundary combination", 0, 0);
    return NULL;
  }
  ora_state* s = (ora_state*)xcalloc(1, sizeof(ora_state));
  s->p = *p;
  s->nx = p->nx;
  s->ny = p->ny;
  s->n = p->nx * p->ny;
  s->ns = p->ns;
  s->T0 = p->T0_K;
  int n = s->n, ns = s->ns;
  double Mmin = 1e300;
  for (int j = 0; j < ns; ++j) Mmin = p->M_gmol[j] < Mmin ? p->M_gmol[j] : Mmin;
  for (int j = 0; j < ns; ++j) {
    s->M[j] = p->M_gmol[j] / Mmin; /* molar masses relative to the lightest, Sec. 2 */
    s->c[j] = 1.0 / sqrt(s->M[j]); /* c_j = sqrt(M0 / M_j), Eq. cx */
  }
  s->mask = (unsigned char*)xcalloc((size_t)n, 1);
  memcpy(s->mask, p->mask, (size_t)n);
  s->p.mask = s->mask;
  s->p.init_X = s->p.init_u = s->p.init_T = s->p.init_Ts = s->p.init_C = NULL;
  s->wall_u = (double*)xcalloc((size_t)2 * n, sizeof(double));
  if (p->wall_u) memcpy(s->wall_u, p->wall_u, sizeof(double) * 2 * (size_t)n);
  s->p.wall_u = s->wall_u;
  s->cls = (int*)xcalloc((size_t)n, sizeof(int));
  size_t np = (size_t)ns * Q * n;
  s->g = (double*)xcalloc(np, sizeof(double));
  s->gn = (double*)xcalloc(np, sizeof(double));
  s->gp = (double*)xcalloc(np, sizeof(double));
  s->Ts = (double*)xcalloc((size_t)n, sizeof(double));
  s->Tsn = (double*)xcalloc((size_t)n, sizeof(double));
  s->rho = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->ux = (double*)xcalloc((size_t)n, sizeof(double));
  s->uy = (double*)xcalloc((size_t)n, sizeof(double));
  s->T = (double*)xcalloc((size_t)n, sizeof(double));
  s->Tg = (double*)xcalloc((size_t)n, sizeof(double));
  s->Cj = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->Tg_prev = (double*)xcalloc((size_t)n, sizeof(double));
  s->Cj_prev = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->divq = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->tau1_prev = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->tau1_cur = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->tau2_cur = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->q = (double*)xcalloc((size_t)n, sizeof(double));
  s->dE = (double*)xcalloc((size_t)n, sizeof(double));
  s->snap = (double*)xcalloc((size_t)(ns + 4) * n, sizeof(double));

  /* Node classes. */
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      int k = x + s->nx * y;
      if (s->mask[k] == 0) {
        if (x == 0 && p->face_bc[0] == F_INLET) s->cls[k] = CL_INLET;
        else if (x == s->nx - 1 && p->face_bc[1] == F_OUTLET) s->cls[k] = CL_OUTLET;
        else s->cls[k] = CL_GAS;
      } else {
        s->cls[k] = CL_SOLID;
      }
    }
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      int k = x + s->nx * y;
      if (s->cls[k] != CL_SOLID) continue;
      for (int i = 1; i < Q; ++i)
        if (cls_at(s, x + EX[i], y + EY[i]) == CL_GAS) s->cls[k] = CL_WALL;
    }
  /* Geometry checks: every gas node needs all 8 neighbours on the lattice; every
   * outlet node copies its upstream gas neighbour. */
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      int k = x + s->nx * y;
      if (s->cls[k] == CL_GAS) {
        for (int i = 1; i < Q; ++i)
          if (node_at(s, x + EX[i], y + EY[i]) < 0) {
            fail(err, errlen, "gas node touches a closed lattice face", x, y);
            ora_destroy(s);
            return NULL;
          }
      } else if (s->cls[k] == CL_OUTLET) {
        if (s->cls[k - 1] != CL_GAS) {
          fail(err, errlen, "outlet node without an upstream gas node", x, y);
          ora_destroy(s);
          return NULL;
        }
      }
    }

  /* Initial state: g*(0) = f^eq of the initial fields, rho_j = C X_j M_j with C = 1
   * unless a concentration field is given;
   * inlet nodes at the inlet state; wall nodes emit rho_w f^eq(1, 0, T_w) with rho_w of
   * the initial fields at the wall node. */
  double tl = 1.0 / (3.0 * s->T0);
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      int k = x + s->nx * y;
      double X[ORA_MAX_NS];
      for (int j = 0; j < ns; ++j) X[j] = p->init_X ? p->init_X[(size_t)j * n + k] : p->X_init[j];
      double ux = p->init_u ? p->init_u[k] : 0.0;
      double uy = p->init_u ? p->init_u[n + k] : 0.0;
      double T = (p->init_T ? p->init_T[k] : p->T_init_K) * tl;
      double Ts = (p->init_Ts ? p->init_Ts[k] : p->T_solid_init_K) * tl;
      double Cn = p->init_C ? p->init_C[k] : 1.0;
      int c = s->cls[k];
      if (c == CL_INLET) {
        for (int j = 0; j < ns; ++j) X[j] = p->X_inlet[j];
        ux = inlet_u(s, y);
        uy = 0.0;
        T = p->T_inlet_K * tl;
        Cn = 1.0;
      }
      if (c == CL_GAS || c == CL_INLET || c == CL_OUTLET) {
        for (int j = 0; j < ns; ++j) {
          double f[Q];
          ora_equilibrium(Cn * X[j] * s->M[j], ux, uy, s->M[j], T, f);
          for (int i = 0; i < Q; ++i) s->g[PIDX(s, j, i, k)] = f[i];
        }
        if (c == CL_GAS) {
          double Xc[ORA_MAX_NS];
          for (int j = 0; j < ns; ++j) {
            Xc[j] = Cn * X[j];
            s->Cj_prev[(size_t)j * n + k] = Cn * X[j];
          }
          s->Tg_prev[k] = T;
          fill_moments_from_fields(s, k, Xc, ux, uy, T);
          for (int j = 0; j < ns; ++j) s->tau1_prev[(size_t)j * n + k] = p->tau1[j];
          if (p->local_tau) {
            double rl[ORA_MAX_NS], t1[ORA_MAX_NS], t2[ORA_MAX_NS];
            for (int j = 0; j < ns; ++j) rl[j] = Xc[j] * s->M[j];
            ora_local_tau(ns, s->M, p->mu, &p->Djk[0][0], rl, T, t1, t2);
            for (int j = 0; j < ns; ++j) s->tau1_prev[(size_t)j * n + k] = t1[j];
          }
        }
      } else {
        s->Ts[k] = Ts;
        if (c == CL_WALL)
          for (int j = 0; j < ns; ++j)
            for (int i = 1; i < Q; ++i)
              if (cls_at(s, x + EX[i], y + EY[i]) == CL_GAS)
                s->g[PIDX(s, j, i, k)] = Cn * X[j] * s->M[j] * wrest(i, Ts);
      }
    }
  memcpy(s->gn, s->g, np * sizeof(double)); /* inlet nodes keep their state in both buffers */
  double mass[ORA_MAX_NS], moles[ORA_MAX_NS];
  ledger_totals(s, &s->E_gas0, &s->H_solid0, mass, moles);
  for (int j = 0; j < ns; ++j) {
    s->mass0[j] = mass[j];
    s->moles0[j] = moles[j];
  }
  pop_totals(s, &s->E_pop0, s->Mpop0);
  return s;
}

void ora_destroy(ora_state* s) {
  if (!s) return;
  free(s->mask);
  free(s->cls);
  free(s->g);
  free(s->gn);
  free(s->gp);
  free(s->Ts);
  free(s->Tsn);
  free(s->rho);
  free(s->ux);
  free(s->uy);
  free(s->T);
  free(s->Tg);
  free(s->Cj);
  free(s->Tg_prev);
  free(s->Cj_prev);
  free(s->divq);
  free(s->tau1_prev);
  free(s->tau1_cur);
  free(s->tau2_cur);
  free(s->wall_u);
  free(s->q);
  free(s->dE);
  free(s->snap);
  free(s);
}

/* ------------------------------------------------------------------------------------
 * Time step
 * ---------------------------------------------------------------------------------- */

/* Step 1: reactive diffusive wall (Sec. 4.3). Count form of the flux balance (reading
 * R11): the mass the wall re-emits per species equals the mass that arrived plus the
 * reaction source m_j = M_j sum_r nu_rj rate_r; the emitted populations are
 * proportional to f^eq(1, 0, T_w) (Eq. BC_g_ji_1) and the wall density follows from the
 * fixed-point iteration of the paper (reading R7: started from the non-reactive wall
 * density, stopped when max_j |d rho_w| <= tol or after the cap). */
static void wall_pass(ora_state* s) {
  int ns = s->ns;
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      int k = x + s->nx * y;
      s->q[k] = 0.0;
      s->dE[k] = 0.0;
      if (s->cls[k] != CL_WALL) continue;
      double Tw = s->Ts[k]; /* wall temperature = solid temperature, Sec. 5 */
      int out[Q] = {0}, arr[Q] = {0};
      for (int i = 1; i < Q; ++i) {
        out[i] = cls_at(s, x + EX[i], y + EY[i]) == CL_GAS;
        arr[i] = cls_at(s, x - EX[i], y - EY[i]) == CL_GAS;
      }
      /* Emitted shape per species: f^eq_j(1, U_w, T_w) (at rest the rest weights), and
       * its sum B_j over the emission directions. */
      double fw[ORA_MAX_NS][Q], B[ORA_MAX_NS];
      for (int j = 0; j < ns; ++j) {
        ora_equilibrium(1.0, s->wall_u[k], s->wall_u[(size_t)s->n + k], s->M[j], Tw, fw[j]);
        B[j] = 0.0;
        for (int i = 1; i < Q; ++i)
          if (out[i]) B[j] += fw[j][i];
      }
      double A[ORA_MAX_NS], Earr = 0.0;
      for (int j = 0; j < ns; ++j) {
        A[j] = 0.0;
        for (int i = 1; i < Q; ++i)
          if (arr[i]) {
            double v = pull(s, s->g, j, i, x, y, 1);
            double d = v - shift_source(s, s->g, j, i, x, y);
            s->D_int += eps_w(s, j, i) * d;
            s->Dm_int[j] += d;
            A[j] += v;
            Earr += 0.5 * s->c[j] * s->c[j] * (EX[i] * EX[i] + EY[i] * EY[i]) * v;
          }
      }
      double rw[ORA_MAX_NS], rate[ORA_MAX_NR] = {0}, m[ORA_MAX_NS];
      int catalytic = s->mask[k] == 2 && s->p.nr > 0;
      for (int j = 0; j < ns; ++j) rw[j] = A[j] / B[j];
      if (catalytic) {
        int conv = 0;
        for (int it = 0; it < s->p.rho_w_maxit; ++it) {
          rates(s, rw, Tw, rate);
          double d = 0.0;
          for (int j = 0; j < ns; ++j) {
            double mj = 0.0;
            for (int r = 0; r < s->p.nr; ++r) mj += s->M[j] * s->p.nu[r][j] * rate[r];
            double nw = (A[j] + mj) / B[j];
            double dd = fabs(nw - rw[j]);
            d = dd > d ? dd : d;
            rw[j] = nw;
          }
          if (d <= s->p.rho_w_tol) {
            conv = 1;
            break;
          }
        }
        if (!conv) s->noconv += 1.0;
        rates(s, rw, Tw, rate);
      }
      double Eout = 0.0, qk = 0.0;
      for (int j = 0; j < ns; ++j) {
        m[j] = 0.0;
        for (int r = 0; r < s->p.nr && catalytic; ++r) m[j] += s->M[j] * s->p.nu[r][j] * rate[r];
        s->M_rxn[j] += m[j];
        for (int i = 1; i < Q; ++i)
          if (out[i]) {
            double w = fw[j][i] * (A[j] + m[j]) / B[j]; /* Eq. BC_gji, count form */
            s->gn[PIDX(s, j, i, k)] = w;
            Eout += 0.5 * s->c[j] * s->c[j] * (EX[i] * EX[i] + EY[i] * EY[i]) * w;
          }
      }
      if (catalytic)
        for (int r = 0; r < s->p.nr; ++r) qk += -(s->p.dH_Jmol[r] / (3.0 * R_GAS * s->T0)) * rate[r];
      s->q[k] = qk;
      s->dE[k] = Eout - Earr;
    }
}

/* Step 2: gas nodes. 2a pull, 2b Prandtl-flux divergence, 2c collision. */
static void gas_pass(ora_state* s) {
  int ns = s->ns, n = s->n;
  double Pr = s->p.Pr;
  /* 2a: streaming with interpolation into every gas node, then g-temperature and
   * concentrations for the correction term. */
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      int k = x + s->nx * y;
      if (s->cls[k] != CL_GAS) continue;
      double gl[ORA_MAX_NS * Q], Cj[ORA_MAX_NS];
      for (int j = 0; j < ns; ++j)
        for (int i = 0; i < Q; ++i) {
          double v = pull(s, s->g, j, i, x, y, 1);
          s->gp[PIDX(s, j, i, k)] = v;
          gl[j * Q + i] = v;
          if (i == 0) continue;
          /* accounts: the pull's departure from the pure shift, and the populations that
           * cross the inlet and outlet faces (taken from inlet/outlet nodes as s1, or
           * lost by this node into them) */
          double s1 = shift_source(s, s->g, j, i, x, y), e = eps_w(s, j, i);
          s->D_int += e * (v - s1);
          s->Dm_int[j] += v - s1;
          int cu = cls_at(s, x - EX[i], y - EY[i]), cd = cls_at(s, x + EX[i], y + EY[i]);
          double own = s->g[PIDX(s, j, i, k)];
          if (cu == CL_INLET) { s->Q_in += e * s1; s->M_in[j] += s1; }
          if (cu == CL_OUTLET) { s->Q_out += e * s1; s->M_out[j] += s1; }
          if (cd == CL_INLET) { s->Q_in -= e * own; s->M_in[j] -= own; }
          if (cd == CL_OUTLET) { s->Q_out -= e * own; s->M_out[j] -= own; }
        }
      s->Tg[k] = g_temperature(ns, s->M, gl, Cj);
      for (int j = 0; j < ns; ++j) s->Cj[(size_t)j * n + k] = Cj[j];
      /* relaxation times of this step: constants, or (reading R18) from the node's
       * pulled (g) densities and g-temperature */
      double t1[ORA_MAX_NS], t2[ORA_MAX_NS];
      for (int j = 0; j < ns; ++j) {
        t1[j] = s->p.tau1[j];
        t2[j] = s->p.tau2[j];
      }
      if (s->p.local_tau) {
        double rl[ORA_MAX_NS];
        for (int j = 0; j < ns; ++j) {
          rl[j] = 0.0;
          for (int i = 0; i < Q; ++i) rl[j] += gl[j * Q + i];
        }
        ora_local_tau(ns, s->M, s->p.mu, &s->p.Djk[0][0], rl, s->Tg[k], t1, t2);
      }
      for (int j = 0; j < ns; ++j) {
        s->tau1_cur[(size_t)j * n + k] = t1[j];
        s->tau2_cur[(size_t)j * n + k] = t2[j];
      }
    }
  /* 2b: divergence of the energy-correction flux q_j = K_j grad T. It is the sum of
   *  - q^Pr_j of Eq. q_Pr, (2 c_pj / Pr - 4 / M_j) tau1_j C_j T grad T with
   *    c_pj = (D + 2) / (2 M_j) (reading R10), and
   *  - the heat-flux part of the lattice-deviation correction the paper refers to but
   *    does not print (Sec. 2, q'): on D2Q9 the product-form equilibrium carries only
   *    tau1_j C_j T grad T / M_j of the kinetic value 4 tau1_j C_j T grad T / M_j, so the
   *    correction adds the missing 3 tau1_j C_j T grad T / M_j (reading R9, a first-order
   *    Chapman-Enskog result; without any energy correction the model has Pr = 4, as the
   *    paper states for its thermal Couette test).
   * K_j = (2 c_pj / Pr - 1 / M_j) tau1_j C_j T. The divergence is the compact
   * second-order conservative difference on the 4 axis neighbours (reading R8: face
   * coefficients are the mean of the two nodes; faces towards non-gas nodes carry no
   * correction flux). The right-hand side of Eq. final_kinetic_equation is taken at time
   * t, so the gradients use the g-temperature, concentrations and tau1 every gas node
   * formed in 2a of this step. Option phi_lagged takes them from the previous time
   * level instead (the moments of the previous step; the initial fields at the first
   * step). */
  const double* Tgv = s->p.phi_lagged ? s->Tg_prev : s->Tg;
  const double* Cjv = s->p.phi_lagged ? s->Cj_prev : s->Cj;
  const double* t1v = s->p.phi_lagged ? s->tau1_prev : s->tau1_cur;
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      int k = x + s->nx * y;
      if (s->cls[k] != CL_GAS) continue;
      for (int j = 0; j < ns; ++j) {
        double dq = 0.0;
        if (s->p.energy_correction) {
          double cp = 2.0 / s->M[j]; /* (D + 2) / (2 M_j), D = 2 */
          double coef = (2.0 * cp / Pr - 1.0 / s->M[j]); /* times tau1 of the node */
          double Kc = coef * t1v[(size_t)j * n + k] * Cjv[(size_t)j * n + k] * Tgv[k];
          for (int i = 1; i <= 4; ++i) {
            int kn = node_at(s, x + EX[i], y + EY[i]);
            if (kn < 0 || s->cls[kn] != CL_GAS) continue;
            double Kn = coef * t1v[(size_t)j * n + kn] * Cjv[(size_t)j * n + kn] * Tgv[kn];
            dq += 0.5 * (Kc + Kn) * (Tgv[kn] - Tgv[k]);
          }
        }
        s->divq[(size_t)j * n + k] = dq;
      }
    }
  /* 2c: collision. */
  for (int k = 0; k < n; ++k) {
    if (s->cls[k] != CL_GAS) continue;
    double gl[ORA_MAX_NS * Q], go[ORA_MAX_NS * Q], dq[ORA_MAX_NS], mom[ORA_MAX_NS + 4];
    for (int j = 0; j < ns; ++j) {
      dq[j] = s->divq[(size_t)j * n + k];
      for (int i = 0; i < Q; ++i) gl[j * Q + i] = s->gp[PIDX(s, j, i, k)];
    }
    double t1[ORA_MAX_NS], t2[ORA_MAX_NS];
    for (int j = 0; j < ns; ++j) {
      t1[j] = s->tau1_cur[(size_t)j * n + k];
      t2[j] = s->tau2_cur[(size_t)j * n + k];
    }
    ora_collide(ns, s->M, t1, t2, gl, dq, go, mom);
    for (int j = 0; j < ns; ++j)
      for (int i = 0; i < Q; ++i) {
        s->gn[PIDX(s, j, i, k)] = go[j * Q + i];
        s->D_col += eps_w(s, j, i) * (go[j * Q + i] - gl[j * Q + i]);
        s->Dm_col[j] += go[j * Q + i] - gl[j * Q + i];
      }
    for (int j = 0; j < ns; ++j) s->rho[(size_t)j * n + k] = mom[j];
    s->ux[k] = mom[ns];
    s->uy[k] = mom[ns + 1];
    s->T[k] = mom[ns + 2];
  }
  /* The moments of this step become the previous time level of the next one. */
  memcpy(s->Tg_prev, s->Tg, sizeof(double) * (size_t)n);
  memcpy(s->Cj_prev, s->Cj, sizeof(double) * (size_t)ns * n);
  memcpy(s->tau1_prev, s->tau1_cur, sizeof(double) * (size_t)ns * n);
  /* Outlet (reading R13; the paper fixes only the inlet): equilibrium at the inlet
   * pressure p = C_in T_in (C_in = 1) with the composition, velocity and temperature of
   * the upstream gas node, so that the outlet gives the open channel its pressure
   * level. */
  double p_out = s->p.T_inlet_K / (3.0 * s->T0);
  for (int k = 0; k < n; ++k)
    if (s->cls[k] == CL_OUTLET) {
      int ku = k - 1;
      double C = 0.0;
      for (int j = 0; j < ns; ++j) C += s->rho[(size_t)j * n + ku] / s->M[j];
      double Cout = p_out / s->T[ku];
      for (int j = 0; j < ns; ++j) {
        double f[Q];
        double rj = s->rho[(size_t)j * n + ku] / s->M[j] / C * Cout * s->M[j];
        ora_equilibrium(rj, s->ux[ku], s->uy[ku], s->M[j], s->T[ku], f);
        for (int i = 0; i < Q; ++i) s->gn[PIDX(s, j, i, k)] = f[i];
      }
    }
}

/* Step 3: explicit FD heat step in the solid (Eq. heat_equation_fd with the 5-point
 * second difference, Eq. heat_equation_fd_2nd_deriv, on each axis). Neighbours that are
 * gas, inlet, outlet or off a closed face add no solid conduction; off a fixed-T face
 * the neighbour is a ghost at T_outer. Wall nodes add the reaction heat and the gas
 * coupling: either the paper's law (Eq. wall_temperature, gas term with the sign that
 * lets heat flow from hot to cold, reading R12) or the exact energy the diffusive wall
 * handed to the gas this step (conservative reading R12). */
static void solid_pass(ora_state* s) {
  double tl = 1.0 / (3.0 * s->T0);
  double Tout = s->p.T_outer_K * tl;
  double as = s->p.alpha_s, rc = s->p.rhocp_s;
  double Qrxn = 0, Qwall = 0, Qcouple = 0, Qfix = 0;
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      int k = x + s->nx * y;
      int c = s->cls[k];
      if (c != CL_WALL && c != CL_SOLID) continue;
      double Tx = s->Ts[k], lap = 0.0, gas_term = 0.0;
      for (int i = 1; i <= 4; ++i) {
        int kn = node_at(s, x + EX[i], y + EY[i]);
        if (kn >= 0) {
          if (s->cls[kn] == CL_WALL || s->cls[kn] == CL_SOLID) lap += s->Ts[kn] - Tx;
          else if (s->cls[kn] == CL_GAS) gas_term += s->T[kn] - Tx;
        } else {
          int face = (i == 1) ? 1 : (i == 3) ? 0 : (i == 2) ? 3 : 2;
          if (s->p.face_bc[face] == F_FIXED_T) {
            lap += Tout - Tx;
            Qfix += rc * as * (Tout - Tx);
          }
        }
      }
      double Tn = Tx + as * lap;
      if (c == CL_WALL) {
        double couple = s->p.coupling == 1 ? s->p.kappa_f * gas_term : -s->dE[k];
        Tn += (s->q[k] + couple) / rc;
        Qrxn += s->q[k];
        Qwall += s->dE[k];
        Qcouple += couple;
      }
      s->Tsn[k] = Tn;
    }
  s->Q_rxn += Qrxn;
  s->Q_wall += Qwall;
  s->Q_couple += Qcouple;
  s->Q_fixedT += Qfix;
}

int ora_step(ora_state* s, int nsteps) {
  for (int t = 0; t < nsteps; ++t) {
    /* All three passes read time level t only: the solid pass runs before the gas pass
     * so that the paper's coupling still sees the gas temperature T(t). */
    wall_pass(s);
    solid_pass(s);
    gas_pass(s);
    double* tmp = s->g;
    s->g = s->gn;
    s->gn = tmp;
    tmp = s->Ts;
    s->Ts = s->Tsn;
    s->Tsn = tmp;
    s->steps += 1.0;
  }
  return 0;
}

/* ------------------------------------------------------------------------------------
 * Outputs
 * ---------------------------------------------------------------------------------- */
int ora_nfields(const ora_state* s) { return 2 * s->ns + 4; }

/* Moment fields at the current time, [field][node]: rho_j, X_j, ux, uy, T (K) on gas
 * nodes and T_s (K) on solid nodes; zero elsewhere. */
void ora_moments(const ora_state* s, double* out) {
  int ns = s->ns, n = s->n;
  double tK = 3.0 * s->T0;
  memset(out, 0, sizeof(double) * (size_t)(2 * ns + 4) * n);
  for (int k = 0; k < n; ++k) {
    if (s->cls[k] == CL_GAS) {
      double C = 0.0;
      for (int j = 0; j < ns; ++j) C += s->rho[(size_t)j * n + k] / s->M[j];
      for (int j = 0; j < ns; ++j) {
        out[(size_t)j * n + k] = s->rho[(size_t)j * n + k];
        out[(size_t)(ns + j) * n + k] = s->rho[(size_t)j * n + k] / s->M[j] / C;
      }
      out[(size_t)(2 * ns) * n + k] = s->ux[k];
      out[(size_t)(2 * ns + 1) * n + k] = s->uy[k];
      out[(size_t)(2 * ns + 2) * n + k] = s->T[k] * tK;
    } else if (s->cls[k] == CL_WALL || s->cls[k] == CL_SOLID) {
      out[(size_t)(2 * ns + 3) * n + k] = s->Ts[k] * tK;
    }
  }
}

void ora_populations(const ora_state* s, double* out) {
  memcpy(out, s->g, sizeof(double) * (size_t)s->ns * Q * s->n);
}

/* The state a step reads (with the energy correction at the current time level): the
 * stored populations g, the solid temperature and the gas mixture temperature T(f) of the
 * previous step (read by the paper's coupling law). NULL arrays are skipped. */
void ora_get_state(const ora_state* s, double* g, double* Ts, double* T) {
  if (g) memcpy(g, s->g, sizeof(double) * (size_t)s->ns * Q * s->n);
  if (Ts) memcpy(Ts, s->Ts, sizeof(double) * (size_t)s->n);
  if (T) memcpy(T, s->T, sizeof(double) * (size_t)s->n);
}

void ora_set_state(ora_state* s, const double* g, const double* Ts, const double* T) {
  if (g) memcpy(s->g, g, sizeof(double) * (size_t)s->ns * Q * s->n);
  if (Ts) memcpy(s->Ts, Ts, sizeof(double) * (size_t)s->n);
  if (T) memcpy(s->T, T, sizeof(double) * (size_t)s->n);
}

/* Gas energy sum_gas (D/2) C T + rho u^2 / 2 from the f-moments plus the energy
 * 1/2 sum c^2 w of the populations the walls have emitted but the gas has not yet
 * pulled in; solid enthalpy sum_solid (rho c_p)_s T_s; per-species mass and moles on
 * the same gas + in-transit basis. Lattice energy units. Counting the in-transit wall
 * emissions makes the totals exact invariants of the on-lattice scheme. */
static void ledger_totals(const ora_state* s, double* E, double* H, double* mass, double* moles) {
  int ns = s->ns, n = s->n;
  double e = 0, h = 0;
  for (int j = 0; j < ns; ++j) mass[j] = moles[j] = 0.0;
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      int k = x + s->nx * y;
      if (s->cls[k] == CL_GAS) {
        double C = 0, r = 0;
        for (int j = 0; j < ns; ++j) {
          double rj = s->rho[(size_t)j * n + k];
          mass[j] += rj;
          moles[j] += rj / s->M[j];
          C += rj / s->M[j];
          r += rj;
        }
        e += C * s->T[k] + 0.5 * r * (s->ux[k] * s->ux[k] + s->uy[k] * s->uy[k]);
      } else if (s->cls[k] == CL_WALL || s->cls[k] == CL_SOLID) {
        h += s->p.rhocp_s * s->Ts[k];
        if (s->cls[k] == CL_WALL)
          for (int j = 0; j < ns; ++j)
            for (int i = 1; i < Q; ++i)
              if (cls_at(s, x + EX[i], y + EY[i]) == CL_GAS) {
                double w = s->g[PIDX(s, j, i, k)];
                mass[j] += w;
                moles[j] += w / s->M[j];
                e += 0.5 * s->c[j] * s->c[j] * (EX[i] * EX[i] + EY[i] * EY[i]) * w;
              }
      }
    }
  *E = e;
  *H = h;
}

/* Ledger (layout in the header). residual = dE_gas + dH_solid - Q_rxn - Q_fixedT; for a
 * closed box it measures the energy the gas scheme itself does not conserve.
 * solid_residual = dH_solid - (Q_rxn + Q_couple + Q_fixedT) is an identity of the FD
 * step. eps_paper is Eq. error_coupling with the heat of reaction 0 measured from the
 * gas-phase change of its first reactant and the gas term taken as internal plus
 * kinetic energy. */
void ora_balance(const ora_state* s, double* out) {
  int ns = s->ns;
  double E, H, mass[ORA_MAX_NS], moles[ORA_MAX_NS];
  ledger_totals(s, &E, &H, mass, moles);
  out[ORA_B_STEPS] = s->steps;
  out[ORA_B_E_GAS] = E;
  out[ORA_B_E_GAS0] = s->E_gas0;
  out[ORA_B_H_SOLID] = H;
  out[ORA_B_H_SOLID0] = s->H_solid0;
  out[ORA_B_Q_RXN] = s->Q_rxn;
  out[ORA_B_Q_WALL] = s->Q_wall;
  out[ORA_B_Q_COUPLE] = s->Q_couple;
  out[ORA_B_Q_FIXEDT] = s->Q_fixedT;
  out[ORA_B_RESIDUAL] = (E - s->E_gas0) + (H - s->H_solid0) - s->Q_rxn - s->Q_fixedT;
  out[ORA_B_SOLID_RESIDUAL] = (H - s->H_solid0) - (s->Q_rxn + s->Q_couple + s->Q_fixedT);
  double eps = 0.0;
  if (s->p.nr > 0) {
    int jr = -1;
    for (int j = 0; j < ns && jr < 0; ++j)
      if (s->p.nu[0][j] < 0) jr = j;
    if (jr >= 0) {
      double dH = s->p.dH_Jmol[0] / (3.0 * R_GAS * s->T0);
      double Qco = -dH * (moles[jr] - s->moles0[jr]) / s->p.nu[0][jr];
      if (Qco != 0.0) eps = ((E - s->E_gas0) + (H - s->H_solid0) - Qco) / Qco;
    }
  }
  out[ORA_B_EPS_PAPER] = eps;
  out[ORA_B_NOCONV] = s->noconv;
  for (int j = 0; j < ns; ++j) {
    out[ORA_B_MASS + j] = mass[j];
    out[ORA_B_MASS + ns + j] = s->mass0[j];
    out[ORA_B_MASS + 2 * ns + j] = moles[j];
    out[ORA_B_MASS + 3 * ns + j] = s->moles0[j];
  }
}

/* Steady-state residual (reading R16, the paper runs fixed step counts): over the
 * fields F in {ux, uy, X_j, T, T_s}, max_F ||F(t) - F(t-K)||_2 / (K max(||F(t) - F_ref||_2,
 * 1e-30)) with F_ref = 0 for u, the inlet composition for X_j and T_inlet for T and T_s.
 * The first call only stores the snapshot and returns +inf. */
double ora_residual(ora_state* s, int K) {
  int ns = s->ns, n = s->n, nf = ns + 4;
  double tl = 1.0 / (3.0 * s->T0);
  double* cur = (double*)xcalloc((size_t)nf * n, sizeof(double));
  double ref[ORA_MAX_NS + 4];
  ref[0] = ref[1] = 0.0;
  for (int j = 0; j < ns; ++j) ref[2 + j] = s->p.X_inlet[j];
  ref[2 + ns] = ref[3 + ns] = s->p.T_inlet_K * tl;
  for (int k = 0; k < n; ++k) {
    int c = s->cls[k];
    if (c == CL_GAS) {
      double C = 0;
      for (int j = 0; j < ns; ++j) C += s->rho[(size_t)j * n + k] / s->M[j];
      cur[k] = s->ux[k];
      cur[(size_t)n + k] = s->uy[k];
      for (int j = 0; j < ns; ++j) cur[(size_t)(2 + j) * n + k] = s->rho[(size_t)j * n + k] / s->M[j] / C;
      cur[(size_t)(2 + ns) * n + k] = s->T[k];
    }
    if (c == CL_WALL || c == CL_SOLID) cur[(size_t)(3 + ns) * n + k] = s->Ts[k];
  }
  double r = INFINITY;
  if (s->have_snap) {
    r = 0.0;
    for (int f = 0; f < nf; ++f) {
      double dn = 0, fn = 0;
      for (int k = 0; k < n; ++k) {
        int c = s->cls[k];
        int on = (f == nf - 1) ? (c == CL_WALL || c == CL_SOLID) : (c == CL_GAS);
        if (!on) continue;
        double a = cur[(size_t)f * n + k], b = s->snap[(size_t)f * n + k];
        dn += (a - b) * (a - b);
        fn += (a - ref[f]) * (a - ref[f]);
      }
      double den = (double)K * (sqrt(fn) > 1e-30 ? sqrt(fn) : 1e-30);
      double rf = sqrt(dn) / den;
      r = rf > r ? rf : r;
    }
  }
  memcpy(s->snap, cur, sizeof(double) * (size_t)nf * n);
  s->have_snap = 1;
  free(cur);
  return r;
}

/* Class counts (gas, inlet, outlet, wall, solid) and the number of non-rest pulls (all
 * species) taken with each stencil so far (none, central, forward, backward, lin_s0,
 * lin_s2). */
void ora_counts(const ora_state* s, long* out) {
  for (int c = 0; c < 5; ++c) out[c] = 0;
  for (int k = 0; k < s->n; ++k) out[s->cls[k]]++;
  for (int c = 0; c < 6; ++c) out[5 + c] = s->st_count[c];
}

void ora_classes(const ora_state* s, int* out) { memcpy(out, s->cls, sizeof(int) * (size_t)s->n); }

/* Inventory of the stored populations: energy sum (1/2) c_j^2 |e_i|^2 g and mass sum g
 * over the post-collision populations of gas nodes and the wall emissions in transit
 * (inlet and outlet nodes are outside the gas). */
static void pop_totals(const ora_state* s, double* E, double* mass) {
  int ns = s->ns;
  double e = 0.0;
  for (int j = 0; j < ns; ++j) mass[j] = 0.0;
  for (int y = 0; y < s->ny; ++y)
    for (int x = 0; x < s->nx; ++x) {
      int k = x + s->nx * y;
      if (s->cls[k] != CL_GAS && s->cls[k] != CL_WALL) continue;
      for (int j = 0; j < ns; ++j)
        for (int i = 0; i < Q; ++i) {
          if (s->cls[k] == CL_WALL && (i == 0 || cls_at(s, x + EX[i], y + EY[i]) != CL_GAS)) continue;
          double g = s->g[PIDX(s, j, i, k)];
          e += eps_w(s, j, i) * g;
          mass[j] += g;
        }
    }
  *E = e;
}

/* Exact accounts of the scheme (layout in the header). One step moves the stored
 * inventory by what the pulls take from inlet/outlet nodes minus what gas nodes stream
 * into them (Q_inlet, Q_outlet), by the departure of every interpolated pull from the
 * pure shift (D_interp: gas pulls and wall arrivals), by the collision's change
 * (D_collision) and by what the walls emit minus what they receive (Q_wall for energy,
 * the reaction production for mass). With the solid's identity, the energy closure
 * dE_pop + dH_solid - Q_rxn - Q_fixedT - Q_inlet - Q_outlet - D_interp - D_collision -
 * D_coupling vanishes to rounding, D_coupling = Q_wall + Q_couple being zero for the
 * conservative coupling. */
void ora_accounts(const ora_state* s, double* out) {
  int ns = s->ns;
  double E, H, mass[ORA_MAX_NS], moles[ORA_MAX_NS], Ep, Mp[ORA_MAX_NS];
  ledger_totals(s, &E, &H, mass, moles);
  pop_totals(s, &Ep, Mp);
  double Dcpl = s->Q_wall + s->Q_couple;
  out[ORA_A_E_POP] = Ep;
  out[ORA_A_E_POP0] = s->E_pop0;
  out[ORA_A_Q_INLET] = s->Q_in;
  out[ORA_A_Q_OUTLET] = s->Q_out;
  out[ORA_A_D_INTERP] = s->D_int;
  out[ORA_A_D_COLLISION] = s->D_col;
  out[ORA_A_D_COUPLING] = Dcpl;
  out[ORA_A_CLOSURE] = (Ep - s->E_pop0) + (H - s->H_solid0) - s->Q_rxn - s->Q_fixedT - s->Q_in - s->Q_out -
                       s->D_int - s->D_col - Dcpl;
  for (int j = 0; j < ns; ++j) {
    double* m = out + ORA_A_MASS;
    m[j] = Mp[j];
    m[ns + j] = s->Mpop0[j];
    m[2 * ns + j] = s->M_in[j];
    m[3 * ns + j] = s->M_out[j];
    m[4 * ns + j] = s->Dm_int[j];
    m[5 * ns + j] = s->Dm_col[j];
    m[6 * ns + j] = s->M_rxn[j];
    m[7 * ns + j] = (Mp[j] - s->Mpop0[j]) - s->M_in[j] - s->M_out[j] - s->Dm_int[j] - s->Dm_col[j] - s->M_rxn[j];
  }
}
