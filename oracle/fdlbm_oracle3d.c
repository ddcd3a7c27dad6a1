/* Plain FP64 CPU oracle of the coupled FD-LBM scheme for catalytic flow on the D3Q19
 * lattice (Kulyk, Berger, Smith, Harting, arXiv:1804.07588; the 3D lattice is the
 * extension the paper announces in Sec. 2, taken here by reading R1b).
 *
 * TEST INFRASTRUCTURE ONLY: the slow reference the CUDA solver's 3D path is checked
 * against. Plain loops over lattice nodes, one pass per step of the algorithm, in the
 * order of the paper's equations; it shares no code with the CUDA solver or with the
 * D2Q9 oracle. The readings (R1..R17) are the D2Q9 oracle's, carried to three
 * dimensions where they depend on D:
 *   R1b  D3Q19 equilibrium: D3Q27 product form of Eq. eq_state_pop with each corner
 *        population folded onto its 3 face diagonals (+), its 3 axis links (-) and the
 *        rest population (+);
 *   R4   psi on D3Q19: +-1 on the +-alpha axis links, -sgn(c_alpha)/8 on the 8 face
 *        diagonals with c_alpha != 0 (over c_j); phi: -1 at rest, 1/(2D) = 1/6 on the
 *        axis links, 0 on diagonals (over c_j^2);
 *   R5   T(f) = T_g + sum_j divq_j / (2 D C), T_g = (E(g) - J^2/rho) / (D C);
 *   R9   the folded product form carries (D - 1) tau1_j C_j T grad T / M_j of the
 *        kinetic heat flux (D + 2) tau1_j C_j T grad T / M_j (first-order
 *        Chapman-Enskog, as for D2Q9 where D - 1 = 1); the energy correction adds the
 *        rest, so K_j = (2 c_pj / Pr - (D - 1) / M_j) tau1_j C_j T and without the
 *        correction the 3D model has Pr = (D + 2) / (D - 1) = 5/2;
 *   R10  c_pj = (D + 2) / (2 M_j).
 *
 * One time step (reading R14), every pass reading time level t only: wall pass
 * (reactive diffusive wall, Sec. 4.3), solid pass (explicit FD heat step with the
 * interface coupling, Sec. 5), gas pass (pull with the off-lattice interpolation of
 * Sec. 4.2 along each link, moments, energy-correction divergence on the 6 axis
 * neighbours from the moments of this step, collision of Eq. final_kinetic_equation).
 */
#include "fdlbm_oracle3d.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define Q ORA3_Q
#define D 3
/* D3Q19 velocities of the lightest species: rest, axis links, face diagonals; the
 * opposite of direction i > 0 is i + 1 for odd i and i - 1 for even i. */
static const int EX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

static const double R_GAS = 8.314462618; /* J/(mol K) */

enum { CL_GAS = 0, CL_INLET = 1, CL_OUTLET = 2, CL_WALL = 3, CL_SOLID = 4 };
enum { F_PERIODIC = 0, F_INLET = 1, F_OUTLET = 2, F_CLOSED = 3, F_FIXED_T = 4 };
enum { ST_NONE = 0, ST_CENTRAL = 1, ST_FORWARD = 2, ST_BACKWARD = 3, ST_LIN_S0 = 4, ST_LIN_S2 = 5 };

struct ora3_state {
  ora3_problem p;
  int nx, ny, nz, n, ns;
  unsigned char* mask;
  int* cls;
  double M[ORA3_MAX_NS], c[ORA3_MAX_NS];
  double T0;
  double* g;        /* [ns][Q][n] post-collision populations and wall emissions */
  double* gn;
  double* gp;       /* [ns][Q][n] pulled populations of gas nodes */
  double* Ts;
  double* Tsn;
  double* rho;      /* [ns][n] */
  double* u;        /* [3][n] */
  double* T;
  double* Tg;
  double* Cj;       /* [ns][n] */
  double* Tg_prev;
  double* Cj_prev;
  double* divq;     /* [ns][n] */
  double* q;
  double* dE;
  double* snap;
  int have_snap;
  double steps;
  double E_gas0, H_solid0, mass0[ORA3_MAX_NS], moles0[ORA3_MAX_NS];
  double Q_rxn, Q_wall, Q_couple, Q_fixedT, noconv;
  /* Exact accounts (ora3_accounts), as in the D2Q9 oracle. */
  double E_pop0, Q_in, Q_out, D_int, D_col;
  double Mpop0[ORA3_MAX_NS], M_in[ORA3_MAX_NS], M_out[ORA3_MAX_NS], Dm_int[ORA3_MAX_NS], Dm_col[ORA3_MAX_NS],
      M_rxn[ORA3_MAX_NS];
  long st_count[6];
};

/* ------------------------------------------------------------------------------------
 * Lattice helpers
 * ---------------------------------------------------------------------------------- */
static int periodic(const ora3_state* s, int axis) { return s->p.face_bc[2 * axis] == F_PERIODIC; }

static int wrap(const ora3_state* s, int axis, int v, int len) {
  if (v >= 0 && v < len) return v;
  if (!periodic(s, axis)) return -1;
  return ((v % len) + len) % len;
}

/* Node index of (x, y, z), wrapped on periodic axes; -1 outside the lattice. */
static int node_at(const ora3_state* s, int x, int y, int z) {
  x = wrap(s, 0, x, s->nx);
  y = wrap(s, 1, y, s->ny);
  z = wrap(s, 2, z, s->nz);
  if (x < 0 || y < 0 || z < 0) return -1;
  return x + s->nx * (y + s->ny * z);
}

static int cls_at(const ora3_state* s, int x, int y, int z) {
  int k = node_at(s, x, y, z);
  return k < 0 ? -1 : s->cls[k];
}

static size_t PIDX(const ora3_state* s, int j, int i, int k) {
  return ((size_t)j * Q + (size_t)i) * (size_t)s->n + (size_t)k;
}

/* Source existence and stencil choice, reading R6, along link i. */
static int source_exists(const ora3_state* s, int x, int y, int z, int i) {
  int c = cls_at(s, x, y, z);
  if (c == CL_GAS || c == CL_INLET || c == CL_OUTLET) return 1;
  if (c == CL_WALL) return cls_at(s, x + EX[i], y + EY[i], z + EZ[i]) == CL_GAS;
  return 0;
}

static int stencil_code(const ora3_state* s, int x, int y, int z, int i) {
  int e2 = source_exists(s, x - 2 * EX[i], y - 2 * EY[i], z - 2 * EZ[i], i);
  int e0 = source_exists(s, x, y, z, i);
  int ep = source_exists(s, x + EX[i], y + EY[i], z + EZ[i], i);
  int e3 = source_exists(s, x - 3 * EX[i], y - 3 * EY[i], z - 3 * EZ[i], i);
  if (e2 && e0) return ST_CENTRAL;
  if (e0 && ep) return ST_FORWARD;
  if (e2 && e3) return ST_BACKWARD;
  if (e0) return ST_LIN_S0;
  if (e2) return ST_LIN_S2;
  return ST_NONE;
}

/* Quadratic upwind interpolation of Sec. 4.2 along one link (Eqs. interpol_bulk,
 * interpol_away, interpol_towards; the linear and none forms of reading R6). The
 * fraction of a link travelled per step is c_j on every link (reading R2). */
static double interp(int code, double c, double s3, double s2, double s1, double s0, double sp) {
  double a = 1.0 - c;
  double d1, d2;
  switch (code) {
    case ST_CENTRAL:
      d1 = (s0 - s2) / 2.0;
      d2 = s0 - 2.0 * s1 + s2;
      break;
    case ST_FORWARD:
      d1 = (4.0 * s0 - sp - 3.0 * s1) / 2.0;
      d2 = -2.0 * s0 + sp + s1;
      break;
    case ST_BACKWARD:
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

static double pull(ora3_state* s, const double* gsrc, int j, int i, int x, int y, int z, int count) {
  int k0 = node_at(s, x, y, z);
  if (i == 0) return gsrc[PIDX(s, j, 0, k0)];
  int code = stencil_code(s, x, y, z, i);
  if (count) s->st_count[code]++;
  int ex = EX[i], ey = EY[i], ez = EZ[i];
  double s1 = gsrc[PIDX(s, j, i, node_at(s, x - ex, y - ey, z - ez))];
  double s0 = 0, s2 = 0, s3 = 0, sp = 0;
  if (code == ST_CENTRAL || code == ST_FORWARD || code == ST_LIN_S0) s0 = gsrc[PIDX(s, j, i, k0)];
  if (code == ST_CENTRAL || code == ST_BACKWARD || code == ST_LIN_S2)
    s2 = gsrc[PIDX(s, j, i, node_at(s, x - 2 * ex, y - 2 * ey, z - 2 * ez))];
  if (code == ST_BACKWARD) s3 = gsrc[PIDX(s, j, i, node_at(s, x - 3 * ex, y - 3 * ey, z - 3 * ez))];
  if (code == ST_FORWARD) sp = gsrc[PIDX(s, j, i, node_at(s, x + ex, y + ey, z + ez))];
  return interp(code, s->c[j], s3, s2, s1, s0, sp);
}

/* The pure-shift value of a pull: population (j, i) of the node x - e_i. */
static double shift_source(const ora3_state* s, const double* gsrc, int j, int i, int x, int y, int z) {
  return gsrc[PIDX(s, j, i, node_at(s, x - EX[i], y - EY[i], z - EZ[i]))];
}

/* Energy weight of population (j, i): (1/2) c_j^2 |e_i|^2. */
static double eps_w(const ora3_state* s, int j, int i) {
  return 0.5 * s->c[j] * s->c[j] * (double)(EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i]);
}

/* ------------------------------------------------------------------------------------
 * Equilibria, correction coefficients, collision
 * ---------------------------------------------------------------------------------- */

double ora3_interp(int code, double c, double s3, double s2, double s1, double s0, double sp) {
  return interp(code, c, s3, s2, s1, s0, sp);
}

void ora3_velocity(int i, int* out3) {
  out3[0] = EX[i];
  out3[1] = EY[i];
  out3[2] = EZ[i];
}

/* One Cartesian factor of the product-form equilibrium (Eq. eq_state_pop, written with
 * the positive sign of reading R1). */
static double wfac(int e, double v, double M, double T) {
  if (e == 0) return 1.0 - M * v * v - T;
  return 0.5 * ((double)e * sqrt(M) * v + M * v * v + T);
}

/* D3Q19 equilibrium by reading R1b, written out as the fold: first the D3Q27 product
 * f27(a, b, c) = rho w(a; ux) w(b; uy) w(c; uz) for every velocity (a, b, c), then every
 * corner value added to the face diagonals it touches and the rest population, and
 * subtracted from the axis links it touches. */
void ora3_equilibrium(double rho, double ux, double uy, double uz, double M, double T, double* f) {
  double f27[3][3][3];
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b)
      for (int c = -1; c <= 1; ++c)
        f27[a + 1][b + 1][c + 1] = rho * wfac(a, ux, M, T) * wfac(b, uy, M, T) * wfac(c, uz, M, T);
  for (int i = 0; i < Q; ++i) f[i] = f27[EX[i] + 1][EY[i] + 1][EZ[i] + 1];
  for (int a = -1; a <= 1; a += 2)
    for (int b = -1; b <= 1; b += 2)
      for (int c = -1; c <= 1; c += 2) {
        double p = f27[a + 1][b + 1][c + 1];
        for (int i = 0; i < Q; ++i) {
          int nz = (EX[i] != 0) + (EY[i] != 0) + (EZ[i] != 0);
          /* does direction i lie on the corner (a, b, c): each non-zero component equal */
          int on = (EX[i] == 0 || EX[i] == a) && (EY[i] == 0 || EY[i] == b) && (EZ[i] == 0 || EZ[i] == c);
          if (!on) continue;
          if (nz == 0) f[i] += p;
          else if (nz == 1) f[i] -= p;
          else f[i] += p;
        }
      }
}

/* Forcing coefficients psi_jialpha on D3Q19 (reading R4). */
void ora3_psi(double c, double* px, double* py, double* pz) {
  for (int i = 0; i < Q; ++i) {
    int nz = (EX[i] != 0) + (EY[i] != 0) + (EZ[i] != 0);
    double* out[3] = {px, py, pz};
    const int e[3] = {EX[i], EY[i], EZ[i]};
    for (int al = 0; al < 3; ++al) {
      double v = 0.0;
      if (nz == 1 && e[al] != 0) v = (double)e[al];
      if (nz == 2 && e[al] != 0) v = -(double)e[al] / 8.0;
      out[al][i] = v / c;
    }
  }
}

/* Energy-only coefficients phi_ji (reading R4): -1 at rest, 1/(2D) on axis links. */
void ora3_phi(double c, double* phi) {
  for (int i = 0; i < Q; ++i) {
    int nz = (EX[i] != 0) + (EY[i] != 0) + (EZ[i] != 0);
    phi[i] = nz == 0 ? -1.0 : (nz == 1 ? 1.0 / (2.0 * D) : 0.0);
    phi[i] /= c * c;
  }
}

/* Corrective diffusion velocity (reading R3), one Cartesian component. */
static double uc(int ns, const double* rho, const double* Ja, const double* tau2, double ua) {
  double num = 0.0, den = 0.0;
  for (int j = 0; j < ns; ++j) {
    num += (Ja[j] - rho[j] * ua) / (tau2[j] + 0.5);
    den += rho[j] / (tau2[j] + 0.5);
  }
  return num / den;
}

/* Moments of pulled g of one node (Eq. moments_of_g, Eq. moments_of_f). */
static void g_moments(int ns, const double* M, const double* g, double* rho, double* J, double* E) {
  for (int j = 0; j < ns; ++j) {
    double c = 1.0 / sqrt(M[j]);
    double r = 0, jx = 0, jy = 0, jz = 0, e = 0;
    for (int i = 0; i < Q; ++i) {
      double v = g[j * Q + i];
      r += v;
      jx += c * EX[i] * v;
      jy += c * EY[i] * v;
      jz += c * EZ[i] * v;
      e += c * c * (EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i]) * v;
    }
    rho[j] = r;
    J[3 * j] = jx;
    J[3 * j + 1] = jy;
    J[3 * j + 2] = jz;
    E[j] = e;
  }
}

static double g_temperature(int ns, const double* M, const double* g, double* Cj_out) {
  double rho[ORA3_MAX_NS], J[3 * ORA3_MAX_NS], E[ORA3_MAX_NS];
  g_moments(ns, M, g, rho, J, E);
  double r = 0, jx = 0, jy = 0, jz = 0, e = 0, C = 0;
  for (int j = 0; j < ns; ++j) {
    r += rho[j];
    jx += J[3 * j];
    jy += J[3 * j + 1];
    jz += J[3 * j + 2];
    e += E[j];
    C += rho[j] / M[j];
    if (Cj_out) Cj_out[j] = rho[j] / M[j];
  }
  return (e - (jx * jx + jy * jy + jz * jz) / r) / (D * C);
}

/* Collision of one gas node, Eq. final_kinetic_equation (dt = 1), with the f-moments
 * of Eq. moments_of_g as in the D2Q9 oracle and D = 3. */
void ora3_collide(int ns, const double* M, const double* tau1, const double* tau2,
                  const double* g, const double* divq, double* gout, double* mom) {
  double rho[ORA3_MAX_NS], J[3 * ORA3_MAX_NS], E[ORA3_MAX_NS];
  g_moments(ns, M, g, rho, J, E);
  double r = 0, jm[3] = {0, 0, 0}, e = 0, C = 0, sdq = 0;
  for (int j = 0; j < ns; ++j) {
    r += rho[j];
    for (int al = 0; al < 3; ++al) jm[al] += J[3 * j + al];
    e += E[j];
    C += rho[j] / M[j];
    sdq += divq[j];
  }
  double u[3], Uc[3], Ja[ORA3_MAX_NS];
  for (int al = 0; al < 3; ++al) u[al] = jm[al] / r;
  double Tg = (e - (jm[0] * jm[0] + jm[1] * jm[1] + jm[2] * jm[2]) / r) / (D * C);
  double T = Tg + sdq / (2.0 * D * C);
  for (int al = 0; al < 3; ++al) {
    for (int j = 0; j < ns; ++j) Ja[j] = J[3 * j + al];
    Uc[al] = uc(ns, rho, Ja, tau2, u[al]);
  }
  for (int j = 0; j < ns; ++j) {
    double c = 1.0 / sqrt(M[j]);
    double a = 1.0 / (2.0 * tau2[j]);
    double uj[3];
    for (int al = 0; al < 3; ++al) uj[al] = u[al];
    if (rho[j] != 0.0) {
      double lim = sqrt((1.0 - T) / M[j]); /* reading R15 */
      for (int al = 0; al < 3; ++al) {
        double Jf = (J[3 * j + al] + a * rho[j] * (u[al] + Uc[al])) / (1.0 + a);
        double v = Jf / rho[j];
        uj[al] = v > lim ? lim : (v < -lim ? -lim : v);
      }
    }
    double feq[Q], fst[Q], px[Q], py[Q], pz[Q], phi[Q];
    ora3_equilibrium(rho[j], u[0], u[1], u[2], M[j], T, feq);
    ora3_equilibrium(rho[j], uj[0], uj[1], uj[2], M[j], T, fst);
    ora3_psi(c, px, py, pz);
    ora3_phi(c, phi);
    double w1 = 2.0 / (1.0 + 2.0 * tau1[j]);
    for (int i = 0; i < Q; ++i) {
      double Psi = (px[i] * Uc[0] + py[i] * Uc[1] + pz[i] * Uc[2]) * rho[j] / tau2[j];
      double Phi = phi[i] * divq[j];
      double gi = g[j * Q + i];
      gout[j * Q + i] = gi - w1 * (gi - fst[i]) - w1 * (tau1[j] / tau2[j]) * (fst[i] - feq[i]) +
                        w1 * tau1[j] * (Psi + Phi);
    }
  }
  if (mom) {
    for (int j = 0; j < ns; ++j) mom[j] = rho[j];
    mom[ns] = u[0];
    mom[ns + 1] = u[1];
    mom[ns + 2] = u[2];
    mom[ns + 3] = T;
    mom[ns + 4] = Tg;
  }
}

/* Surface kinetics (reading R11), lattice moles per wall node per step. */
static void rates(const ora3_state* s, const double* rho_w, double Tw, double* rate) {
  int ns = s->ns;
  double Cw[ORA3_MAX_NS], Ct = 0;
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

/* Rest-equilibrium weight of direction i at temperature T (f^eq(1, 0, T)). */
static double wrest(int i, double T) {
  double f[Q];
  ora3_equilibrium(1.0, 0.0, 0.0, 0.0, 1.0, T, f);
  return f[i];
}

/* ------------------------------------------------------------------------------------
 * Set-up
 * ---------------------------------------------------------------------------------- */
static void* xcalloc(size_t n, size_t sz) {
  void* p = calloc(n ? n : 1, sz);
  if (!p) {
    fprintf(stderr, "oracle3d: out of memory\n");
    abort();
  }
  return p;
}

static void fail(char* err, int errlen, const char* msg, int x, int y, int z) {
  if (err && errlen > 0) snprintf(err, (size_t)errlen, "%s at (%d,%d,%d)", msg, x, y, z);
}

static void ledger_totals(const ora3_state* s, double* E, double* H, double* mass, double* moles);
static void pop_totals(const ora3_state* s, double* E, double* mass);

ora3_state* ora3_create(const ora3_problem* p, char* err, int errlen) {
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->ns < 1 || p->ns > ORA3_MAX_NS || p->nr < 0 ||
      p->nr > ORA3_MAX_NR) {
    fail(err, errlen, "bad sizes", p->nx, p->ny, p->nz);
    return NULL;
  }
  for (int a = 0; a < 3; ++a)
    if ((p->face_bc[2 * a] == F_PERIODIC) != (p->face_bc[2 * a + 1] == F_PERIODIC)) {
      fail(err, errlen, "periodic faces come in pairs", a, 0, 0);
      return NULL;
    }
  for (int f = 0; f < 6; ++f)
    if ((p->face_bc[f] == F_INLET && f != 0) || (p->face_bc[f] == F_OUTLET && f != 1)) {
      fail(err, errlen, "inlet only on x-, outlet only on x+", f, 0, 0);
      return NULL;
    }
  ora3_state* s = (ora3_state*)xcalloc(1, sizeof(ora3_state));
  s->p = *p;
  s->nx = p->nx;
  s->ny = p->ny;
  s->nz = p->nz;
  s->n = p->nx * p->ny * p->nz;
  s->ns = p->ns;
  s->T0 = p->T0_K;
  int n = s->n, ns = s->ns;
  double Mmin = 1e300;
  for (int j = 0; j < ns; ++j) Mmin = p->M_gmol[j] < Mmin ? p->M_gmol[j] : Mmin;
  for (int j = 0; j < ns; ++j) {
    s->M[j] = p->M_gmol[j] / Mmin;
    s->c[j] = 1.0 / sqrt(s->M[j]);
  }
  s->mask = (unsigned char*)xcalloc((size_t)n, 1);
  memcpy(s->mask, p->mask, (size_t)n);
  s->p.mask = s->mask;
  s->p.init_X = s->p.init_u = s->p.init_T = s->p.init_Ts = s->p.init_C = NULL;
  s->cls = (int*)xcalloc((size_t)n, sizeof(int));
  size_t np = (size_t)ns * Q * n;
  s->g = (double*)xcalloc(np, sizeof(double));
  s->gn = (double*)xcalloc(np, sizeof(double));
  s->gp = (double*)xcalloc(np, sizeof(double));
  s->Ts = (double*)xcalloc((size_t)n, sizeof(double));
  s->Tsn = (double*)xcalloc((size_t)n, sizeof(double));
  s->rho = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->u = (double*)xcalloc((size_t)3 * n, sizeof(double));
  s->T = (double*)xcalloc((size_t)n, sizeof(double));
  s->Tg = (double*)xcalloc((size_t)n, sizeof(double));
  s->Cj = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->Tg_prev = (double*)xcalloc((size_t)n, sizeof(double));
  s->Cj_prev = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->divq = (double*)xcalloc((size_t)ns * n, sizeof(double));
  s->q = (double*)xcalloc((size_t)n, sizeof(double));
  s->dE = (double*)xcalloc((size_t)n, sizeof(double));
  s->snap = (double*)xcalloc((size_t)(ns + 5) * n, sizeof(double));

  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        int k = x + s->nx * (y + s->ny * z);
        if (s->mask[k] == 0) {
          if (x == 0 && p->face_bc[0] == F_INLET) s->cls[k] = CL_INLET;
          else if (x == s->nx - 1 && p->face_bc[1] == F_OUTLET) s->cls[k] = CL_OUTLET;
          else s->cls[k] = CL_GAS;
        } else {
          s->cls[k] = CL_SOLID;
        }
      }
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        int k = x + s->nx * (y + s->ny * z);
        if (s->cls[k] != CL_SOLID) continue;
        for (int i = 1; i < Q; ++i)
          if (cls_at(s, x + EX[i], y + EY[i], z + EZ[i]) == CL_GAS) s->cls[k] = CL_WALL;
      }
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        int k = x + s->nx * (y + s->ny * z);
        if (s->cls[k] == CL_GAS) {
          for (int i = 1; i < Q; ++i)
            if (node_at(s, x + EX[i], y + EY[i], z + EZ[i]) < 0) {
              fail(err, errlen, "gas node touches a closed lattice face", x, y, z);
              ora3_destroy(s);
              return NULL;
            }
        } else if (s->cls[k] == CL_OUTLET && s->cls[k - 1] != CL_GAS) {
          fail(err, errlen, "outlet node without an upstream gas node", x, y, z);
          ora3_destroy(s);
          return NULL;
        }
      }

  /* Initial state as in the D2Q9 oracle: equilibrium of the initial fields on gas,
   * inlet (inlet state) and outlet nodes; wall nodes emit rho_w f^eq(1, 0, T_s). */
  double tl = 1.0 / (3.0 * s->T0);
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        int k = x + s->nx * (y + s->ny * z);
        double X[ORA3_MAX_NS], u[3];
        for (int j = 0; j < ns; ++j) X[j] = p->init_X ? p->init_X[(size_t)j * n + k] : p->X_init[j];
        for (int al = 0; al < 3; ++al) u[al] = p->init_u ? p->init_u[(size_t)al * n + k] : 0.0;
        double T = (p->init_T ? p->init_T[k] : p->T_init_K) * tl;
        double Ts = (p->init_Ts ? p->init_Ts[k] : p->T_solid_init_K) * tl;
        double Cn = p->init_C ? p->init_C[k] : 1.0;
        int c = s->cls[k];
        if (c == CL_INLET) {
          for (int j = 0; j < ns; ++j) X[j] = p->X_inlet[j];
          u[0] = p->u_inlet;
          u[1] = u[2] = 0.0;
          T = p->T_inlet_K * tl;
          Cn = 1.0;
        }
        if (c == CL_GAS || c == CL_INLET || c == CL_OUTLET) {
          for (int j = 0; j < ns; ++j) {
            double f[Q];
            ora3_equilibrium(Cn * X[j] * s->M[j], u[0], u[1], u[2], s->M[j], T, f);
            for (int i = 0; i < Q; ++i) s->g[PIDX(s, j, i, k)] = f[i];
          }
          if (c == CL_GAS) {
            for (int j = 0; j < ns; ++j) {
              s->Cj_prev[(size_t)j * n + k] = Cn * X[j];
              s->rho[(size_t)j * n + k] = Cn * X[j] * s->M[j];
            }
            s->Tg_prev[k] = T;
            for (int al = 0; al < 3; ++al) s->u[(size_t)al * n + k] = u[al];
            s->T[k] = T;
          }
        } else {
          s->Ts[k] = Ts;
          if (c == CL_WALL)
            for (int j = 0; j < ns; ++j)
              for (int i = 1; i < Q; ++i)
                if (cls_at(s, x + EX[i], y + EY[i], z + EZ[i]) == CL_GAS)
                  s->g[PIDX(s, j, i, k)] = Cn * X[j] * s->M[j] * wrest(i, Ts);
        }
      }
  memcpy(s->gn, s->g, np * sizeof(double));
  double mass[ORA3_MAX_NS], moles[ORA3_MAX_NS];
  ledger_totals(s, &s->E_gas0, &s->H_solid0, mass, moles);
  for (int j = 0; j < ns; ++j) {
    s->mass0[j] = mass[j];
    s->moles0[j] = moles[j];
  }
  pop_totals(s, &s->E_pop0, s->Mpop0);
  return s;
}

void ora3_destroy(ora3_state* s) {
  if (!s) return;
  free(s->mask);
  free(s->cls);
  free(s->g);
  free(s->gn);
  free(s->gp);
  free(s->Ts);
  free(s->Tsn);
  free(s->rho);
  free(s->u);
  free(s->T);
  free(s->Tg);
  free(s->Cj);
  free(s->Tg_prev);
  free(s->Cj_prev);
  free(s->divq);
  free(s->q);
  free(s->dE);
  free(s->snap);
  free(s);
}

/* ------------------------------------------------------------------------------------
 * Time step
 * ---------------------------------------------------------------------------------- */

/* Step 1: reactive diffusive wall (Sec. 4.3; count form and iteration, readings R7,
 * R11), as in the D2Q9 oracle with the 18 links of D3Q19. */
static void wall_pass(ora3_state* s) {
  int ns = s->ns;
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        int k = x + s->nx * (y + s->ny * z);
        s->q[k] = 0.0;
        s->dE[k] = 0.0;
        if (s->cls[k] != CL_WALL) continue;
        double Tw = s->Ts[k];
        int out[Q] = {0}, arr[Q] = {0};
        double wr[Q], B = 0.0;
        ora3_equilibrium(1.0, 0.0, 0.0, 0.0, 1.0, Tw, wr); /* f^eq(1, 0, T_w) */
        for (int i = 1; i < Q; ++i) {
          out[i] = cls_at(s, x + EX[i], y + EY[i], z + EZ[i]) == CL_GAS;
          arr[i] = cls_at(s, x - EX[i], y - EY[i], z - EZ[i]) == CL_GAS;
          if (out[i]) B += wr[i];
        }
        double A[ORA3_MAX_NS], Earr = 0.0;
        for (int j = 0; j < ns; ++j) {
          A[j] = 0.0;
          for (int i = 1; i < Q; ++i)
            if (arr[i]) {
              double v = pull(s, s->g, j, i, x, y, z, 1);
              double d = v - shift_source(s, s->g, j, i, x, y, z);
              s->D_int += eps_w(s, j, i) * d;
              s->Dm_int[j] += d;
              A[j] += v;
              Earr += 0.5 * s->c[j] * s->c[j] * (EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i]) * v;
            }
        }
        double rw[ORA3_MAX_NS], rate[ORA3_MAX_NR] = {0}, m[ORA3_MAX_NS];
        int catalytic = s->mask[k] == 2 && s->p.nr > 0;
        for (int j = 0; j < ns; ++j) rw[j] = A[j] / B;
        if (catalytic) {
          int conv = 0;
          for (int it = 0; it < s->p.rho_w_maxit; ++it) {
            rates(s, rw, Tw, rate);
            double d = 0.0;
            for (int j = 0; j < ns; ++j) {
              double mj = 0.0;
              for (int r = 0; r < s->p.nr; ++r) mj += s->M[j] * s->p.nu[r][j] * rate[r];
              double nw = (A[j] + mj) / B;
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
              double w = wr[i] * (A[j] + m[j]) / B; /* Eq. BC_gji, count form */
              s->gn[PIDX(s, j, i, k)] = w;
              Eout += 0.5 * s->c[j] * s->c[j] * (EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i]) * w;
            }
        }
        if (catalytic)
          for (int r = 0; r < s->p.nr; ++r) qk += -(s->p.dH_Jmol[r] / (3.0 * R_GAS * s->T0)) * rate[r];
        s->q[k] = qk;
        s->dE[k] = Eout - Earr;
      }
}

/* Step 2: gas nodes (pull, energy-correction divergence, collision, outlet). */
static void gas_pass(ora3_state* s) {
  int ns = s->ns, n = s->n;
  double Pr = s->p.Pr;
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        int k = x + s->nx * (y + s->ny * z);
        if (s->cls[k] != CL_GAS) continue;
        double gl[ORA3_MAX_NS * Q], Cj[ORA3_MAX_NS];
        for (int j = 0; j < ns; ++j)
          for (int i = 0; i < Q; ++i) {
            double v = pull(s, s->g, j, i, x, y, z, 1);
            s->gp[PIDX(s, j, i, k)] = v;
            gl[j * Q + i] = v;
            if (i == 0) continue;
            /* accounts (see the D2Q9 oracle) */
            double s1 = shift_source(s, s->g, j, i, x, y, z), e = eps_w(s, j, i);
            s->D_int += e * (v - s1);
            s->Dm_int[j] += v - s1;
            int cu = cls_at(s, x - EX[i], y - EY[i], z - EZ[i]), cd = cls_at(s, x + EX[i], y + EY[i], z + EZ[i]);
            double own = s->g[PIDX(s, j, i, k)];
            if (cu == CL_INLET) { s->Q_in += e * s1; s->M_in[j] += s1; }
            if (cu == CL_OUTLET) { s->Q_out += e * s1; s->M_out[j] += s1; }
            if (cd == CL_INLET) { s->Q_in -= e * own; s->M_in[j] -= own; }
            if (cd == CL_OUTLET) { s->Q_out -= e * own; s->M_out[j] -= own; }
          }
        s->Tg[k] = g_temperature(ns, s->M, gl, Cj);
        for (int j = 0; j < ns; ++j) s->Cj[(size_t)j * n + k] = Cj[j];
      }
  /* Energy-correction divergence (readings R8, R9, R10 with D = 3) on the 6 axis
   * neighbours from the moments of this step (option phi_lagged: of the previous time
   * level); faces to non-gas nodes carry no flux. */
  const double* Tgv = s->p.phi_lagged ? s->Tg_prev : s->Tg;
  const double* Cjv = s->p.phi_lagged ? s->Cj_prev : s->Cj;
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        int k = x + s->nx * (y + s->ny * z);
        if (s->cls[k] != CL_GAS) continue;
        for (int j = 0; j < ns; ++j) {
          double dq = 0.0;
          if (s->p.energy_correction) {
            double cp = (D + 2.0) / (2.0 * s->M[j]);
            double coef = (2.0 * cp / Pr - (D - 1.0) / s->M[j]) * s->p.tau1[j];
            double Kc = coef * Cjv[(size_t)j * n + k] * Tgv[k];
            for (int i = 1; i <= 6; ++i) {
              int kn = node_at(s, x + EX[i], y + EY[i], z + EZ[i]);
              if (kn < 0 || s->cls[kn] != CL_GAS) continue;
              double Kn = coef * Cjv[(size_t)j * n + kn] * Tgv[kn];
              dq += 0.5 * (Kc + Kn) * (Tgv[kn] - Tgv[k]);
            }
          }
          s->divq[(size_t)j * n + k] = dq;
        }
      }
  for (int k = 0; k < n; ++k) {
    if (s->cls[k] != CL_GAS) continue;
    double gl[ORA3_MAX_NS * Q], go[ORA3_MAX_NS * Q], dq[ORA3_MAX_NS], mom[ORA3_MAX_NS + 5];
    for (int j = 0; j < ns; ++j) {
      dq[j] = s->divq[(size_t)j * n + k];
      for (int i = 0; i < Q; ++i) gl[j * Q + i] = s->gp[PIDX(s, j, i, k)];
    }
    ora3_collide(ns, s->M, s->p.tau1, s->p.tau2, gl, dq, go, mom);
    for (int j = 0; j < ns; ++j)
      for (int i = 0; i < Q; ++i) {
        s->gn[PIDX(s, j, i, k)] = go[j * Q + i];
        s->D_col += eps_w(s, j, i) * (go[j * Q + i] - gl[j * Q + i]);
        s->Dm_col[j] += go[j * Q + i] - gl[j * Q + i];
      }
    for (int j = 0; j < ns; ++j) s->rho[(size_t)j * n + k] = mom[j];
    for (int al = 0; al < 3; ++al) s->u[(size_t)al * n + k] = mom[ns + al];
    s->T[k] = mom[ns + 3];
  }
  memcpy(s->Tg_prev, s->Tg, sizeof(double) * (size_t)n);
  memcpy(s->Cj_prev, s->Cj, sizeof(double) * (size_t)ns * n);
  /* Outlet (reading R13): equilibrium at the inlet pressure with the composition,
   * velocity and temperature of the upstream gas node. */
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
        ora3_equilibrium(rj, s->u[ku], s->u[(size_t)n + ku], s->u[(size_t)2 * n + ku], s->M[j], s->T[ku], f);
        for (int i = 0; i < Q; ++i) s->gn[PIDX(s, j, i, k)] = f[i];
      }
    }
}

/* Step 3: explicit FD heat step in the solid, 7-point second difference (Eqs.
 * heat_equation_fd, heat_equation_fd_2nd_deriv on each of the 3 axes), with the
 * interface coupling of reading R12 and the reaction heat on wall nodes. */
static void solid_pass(ora3_state* s) {
  double tl = 1.0 / (3.0 * s->T0);
  double Tout = s->p.T_outer_K * tl;
  double as = s->p.alpha_s, rc = s->p.rhocp_s;
  double Qrxn = 0, Qwall = 0, Qcouple = 0, Qfix = 0;
  static const int FACE[7] = {-1, 1, 0, 3, 2, 5, 4}; /* face left through axis link i */
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        int k = x + s->nx * (y + s->ny * z);
        int c = s->cls[k];
        if (c != CL_WALL && c != CL_SOLID) continue;
        double Tx = s->Ts[k], lap = 0.0, gas_term = 0.0;
        for (int i = 1; i <= 6; ++i) {
          int kn = node_at(s, x + EX[i], y + EY[i], z + EZ[i]);
          if (kn >= 0) {
            if (s->cls[kn] == CL_WALL || s->cls[kn] == CL_SOLID) lap += s->Ts[kn] - Tx;
            else if (s->cls[kn] == CL_GAS) gas_term += s->T[kn] - Tx;
          } else if (s->p.face_bc[FACE[i]] == F_FIXED_T) {
            lap += Tout - Tx;
            Qfix += rc * as * (Tout - Tx);
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

int ora3_step(ora3_state* s, int nsteps) {
  for (int t = 0; t < nsteps; ++t) {
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
int ora3_nfields(const ora3_state* s) { return 2 * s->ns + 5; }

void ora3_moments(const ora3_state* s, double* out) {
  int ns = s->ns, n = s->n;
  double tK = 3.0 * s->T0;
  memset(out, 0, sizeof(double) * (size_t)(2 * ns + 5) * n);
  for (int k = 0; k < n; ++k) {
    if (s->cls[k] == CL_GAS) {
      double C = 0.0;
      for (int j = 0; j < ns; ++j) C += s->rho[(size_t)j * n + k] / s->M[j];
      for (int j = 0; j < ns; ++j) {
        out[(size_t)j * n + k] = s->rho[(size_t)j * n + k];
        out[(size_t)(ns + j) * n + k] = s->rho[(size_t)j * n + k] / s->M[j] / C;
      }
      for (int al = 0; al < 3; ++al) out[(size_t)(2 * ns + al) * n + k] = s->u[(size_t)al * n + k];
      out[(size_t)(2 * ns + 3) * n + k] = s->T[k] * tK;
    } else if (s->cls[k] == CL_WALL || s->cls[k] == CL_SOLID) {
      out[(size_t)(2 * ns + 4) * n + k] = s->Ts[k] * tK;
    }
  }
}

void ora3_populations(const ora3_state* s, double* out) {
  memcpy(out, s->g, sizeof(double) * (size_t)s->ns * Q * s->n);
}

/* The state the next step reads: stored populations, solid temperature and the gas
 * mixture temperature of the last step (read by the paper's coupling law). */
void ora3_get_state(const ora3_state* s, double* g, double* Ts, double* T) {
  if (g) memcpy(g, s->g, sizeof(double) * (size_t)s->ns * Q * s->n);
  if (Ts) memcpy(Ts, s->Ts, sizeof(double) * (size_t)s->n);
  if (T) memcpy(T, s->T, sizeof(double) * (size_t)s->n);
}

void ora3_set_state(ora3_state* s, const double* g, const double* Ts, const double* T) {
  if (g) memcpy(s->g, g, sizeof(double) * (size_t)s->ns * Q * s->n);
  if (Ts) memcpy(s->Ts, Ts, sizeof(double) * (size_t)s->n);
  if (T) memcpy(s->T, T, sizeof(double) * (size_t)s->n);
}

/* Gas energy sum (D/2) C T + rho u^2 / 2 plus the in-transit wall emissions; solid
 * enthalpy; species mass and moles (as in the D2Q9 oracle). */
static void ledger_totals(const ora3_state* s, double* E, double* H, double* mass, double* moles) {
  int ns = s->ns, n = s->n;
  double e = 0, h = 0;
  for (int j = 0; j < ns; ++j) mass[j] = moles[j] = 0.0;
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        int k = x + s->nx * (y + s->ny * z);
        if (s->cls[k] == CL_GAS) {
          double C = 0, r = 0, u2 = 0;
          for (int j = 0; j < ns; ++j) {
            double rj = s->rho[(size_t)j * n + k];
            mass[j] += rj;
            moles[j] += rj / s->M[j];
            C += rj / s->M[j];
            r += rj;
          }
          for (int al = 0; al < 3; ++al) u2 += s->u[(size_t)al * n + k] * s->u[(size_t)al * n + k];
          e += 0.5 * D * C * s->T[k] + 0.5 * r * u2;
        } else if (s->cls[k] == CL_WALL || s->cls[k] == CL_SOLID) {
          h += s->p.rhocp_s * s->Ts[k];
          if (s->cls[k] == CL_WALL)
            for (int j = 0; j < ns; ++j)
              for (int i = 1; i < Q; ++i)
                if (cls_at(s, x + EX[i], y + EY[i], z + EZ[i]) == CL_GAS) {
                  double w = s->g[PIDX(s, j, i, k)];
                  mass[j] += w;
                  moles[j] += w / s->M[j];
                  e += 0.5 * s->c[j] * s->c[j] * (EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i]) * w;
                }
        }
      }
  *E = e;
  *H = h;
}

void ora3_balance(const ora3_state* s, double* out) {
  int ns = s->ns;
  double E, H, mass[ORA3_MAX_NS], moles[ORA3_MAX_NS];
  ledger_totals(s, &E, &H, mass, moles);
  out[ORA3_B_STEPS] = s->steps;
  out[ORA3_B_E_GAS] = E;
  out[ORA3_B_E_GAS0] = s->E_gas0;
  out[ORA3_B_H_SOLID] = H;
  out[ORA3_B_H_SOLID0] = s->H_solid0;
  out[ORA3_B_Q_RXN] = s->Q_rxn;
  out[ORA3_B_Q_WALL] = s->Q_wall;
  out[ORA3_B_Q_COUPLE] = s->Q_couple;
  out[ORA3_B_Q_FIXEDT] = s->Q_fixedT;
  out[ORA3_B_RESIDUAL] = (E - s->E_gas0) + (H - s->H_solid0) - s->Q_rxn - s->Q_fixedT;
  out[ORA3_B_SOLID_RESIDUAL] = (H - s->H_solid0) - (s->Q_rxn + s->Q_couple + s->Q_fixedT);
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
  out[ORA3_B_EPS_PAPER] = eps;
  out[ORA3_B_NOCONV] = s->noconv;
  for (int j = 0; j < ns; ++j) {
    out[ORA3_B_MASS + j] = mass[j];
    out[ORA3_B_MASS + ns + j] = s->mass0[j];
    out[ORA3_B_MASS + 2 * ns + j] = moles[j];
    out[ORA3_B_MASS + 3 * ns + j] = s->moles0[j];
  }
}

/* Steady-state residual (reading R16) over ux, uy, uz, X_j, T, T_s. */
double ora3_residual(ora3_state* s, int K) {
  int ns = s->ns, n = s->n, nf = ns + 5;
  double tl = 1.0 / (3.0 * s->T0);
  double* cur = (double*)xcalloc((size_t)nf * n, sizeof(double));
  double ref[ORA3_MAX_NS + 5];
  ref[0] = ref[1] = ref[2] = 0.0;
  for (int j = 0; j < ns; ++j) ref[3 + j] = s->p.X_inlet[j];
  ref[3 + ns] = ref[4 + ns] = s->p.T_inlet_K * tl;
  for (int k = 0; k < n; ++k) {
    int c = s->cls[k];
    if (c == CL_GAS) {
      double C = 0;
      for (int j = 0; j < ns; ++j) C += s->rho[(size_t)j * n + k] / s->M[j];
      for (int al = 0; al < 3; ++al) cur[(size_t)al * n + k] = s->u[(size_t)al * n + k];
      for (int j = 0; j < ns; ++j) cur[(size_t)(3 + j) * n + k] = s->rho[(size_t)j * n + k] / s->M[j] / C;
      cur[(size_t)(3 + ns) * n + k] = s->T[k];
    }
    if (c == CL_WALL || c == CL_SOLID) cur[(size_t)(4 + ns) * n + k] = s->Ts[k];
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

void ora3_counts(const ora3_state* s, long* out) {
  for (int c = 0; c < 5; ++c) out[c] = 0;
  for (int k = 0; k < s->n; ++k) out[s->cls[k]]++;
  for (int c = 0; c < 6; ++c) out[5 + c] = s->st_count[c];
}

void ora3_classes(const ora3_state* s, int* out) { memcpy(out, s->cls, sizeof(int) * (size_t)s->n); }

/* Inventory of the stored populations (gas nodes and wall emissions in transit). */
static void pop_totals(const ora3_state* s, double* E, double* mass) {
  int ns = s->ns;
  double e = 0.0;
  for (int j = 0; j < ns; ++j) mass[j] = 0.0;
  for (int z = 0; z < s->nz; ++z)
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x) {
        int k = x + s->nx * (y + s->ny * z);
        if (s->cls[k] != CL_GAS && s->cls[k] != CL_WALL) continue;
        for (int j = 0; j < ns; ++j)
          for (int i = 0; i < Q; ++i) {
            if (s->cls[k] == CL_WALL && (i == 0 || cls_at(s, x + EX[i], y + EY[i], z + EZ[i]) != CL_GAS)) continue;
            double g = s->g[PIDX(s, j, i, k)];
            e += eps_w(s, j, i) * g;
            mass[j] += g;
          }
      }
  *E = e;
}

/* Exact accounts (layout ORA3_A_*, the D2Q9 oracle's). */
void ora3_accounts(const ora3_state* s, double* out) {
  int ns = s->ns;
  double E, H, mass[ORA3_MAX_NS], moles[ORA3_MAX_NS], Ep, Mp[ORA3_MAX_NS];
  ledger_totals(s, &E, &H, mass, moles);
  pop_totals(s, &Ep, Mp);
  double Dcpl = s->Q_wall + s->Q_couple;
  out[ORA3_A_E_POP] = Ep;
  out[ORA3_A_E_POP0] = s->E_pop0;
  out[ORA3_A_Q_INLET] = s->Q_in;
  out[ORA3_A_Q_OUTLET] = s->Q_out;
  out[ORA3_A_D_INTERP] = s->D_int;
  out[ORA3_A_D_COLLISION] = s->D_col;
  out[ORA3_A_D_COUPLING] = Dcpl;
  out[ORA3_A_CLOSURE] = (Ep - s->E_pop0) + (H - s->H_solid0) - s->Q_rxn - s->Q_fixedT - s->Q_in - s->Q_out -
                        s->D_int - s->D_col - Dcpl;
  double* m = out + ORA3_A_MASS;
  for (int j = 0; j < ns; ++j) {
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
