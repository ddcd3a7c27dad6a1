// Host side of the solver library: the C ABI of include/fdlbm.h.
//
// fdlbm_create validates the problem, converts units (Sec. 4.1: lattice temperature
// T / (3 T0), molar masses relative to the lightest species, c_j = 1/sqrt(M_j)),
// classifies nodes, precomputes the streaming stencil of every pull (Sec. 4.2 and the
// near-wall readings), builds the solid-node list (interface wall nodes first) and
// initialises the device state. Kernels live in fdlbm_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "fdlbm_internal.h"

using namespace fdlbm;

namespace {

thread_local std::string g_err = "no error";

fdlbm_status fail(fdlbm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

constexpr double R_GAS = 8.314462618;
constexpr int HEX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int HEY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

struct Alloc {
  void* p;
  size_t bytes;
};

}  // namespace

struct fdlbm_handle {
  DevParams P{};
  DevState S{};
  int cur = 0;                // buffer holding g*(t)
  int64_t steps = 0;
  int64_t steps_at_residual = 0;
  bool have_snap = false;
  bool mom_fresh = true;      // S.mom holds the moments of the current time
  cudaStream_t stream = nullptr;
  int device = 0;
  void* (*ualloc)(size_t, void*) = nullptr;
  void (*ufree)(void*, size_t, void*) = nullptr;
  void* uctx = nullptr;
  std::vector<Alloc> allocs;
  size_t bytes = 0;
  float* out_buf = nullptr;   // staging for host copies of outputs
  // host-side description kept for re-initialisation and outputs
  int nx = 0, ny = 0, ns = 0;
  int dim = 2, nz = 1;        // D2Q9 (2) or D3Q19 (3)
  std::vector<uint32_t> code;
  std::vector<double> X_init, X_inlet, inlet_u;
  double T0 = 0, T_init_lat = 0, T_inlet_lat = 0, Ts_init_lat = 0;
  double T_st = 0;  // reference temperature of the stored deviations (a multiple of 2^-12)
  double heat0 = 0;           // -dH / (3 R T0) of reaction 0
  int eps_species = -1, eps_nu = 0;
  double E0 = 0, H0 = 0, mass0[MAX_NS] = {}, moles0[MAX_NS] = {};
  double E_pop0 = 0;          // energy of the stored populations at the start (exact accounts)
  int64_t counts[5] = {};
  std::vector<int4> blocks_host;  // step-kernel block descriptors (for batches)
  int64_t stencil_counts[6] = {};
  // optional kernel timing: three events per step (before solid, between, after gas)
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  size_t events_used = 0;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

fdlbm_status cuda_fail(cudaError_t e, const char* what) {
  return fail(FDLBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                           \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

fdlbm_status dalloc(fdlbm_handle* h, size_t bytes, void** out) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (h->ualloc) {
    p = h->ualloc(bytes, h->uctx);
    if (!p) return fail(FDLBM_ENOMEM, "caller allocator returned NULL for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(FDLBM_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  h->allocs.push_back({p, bytes});
  h->bytes += bytes;
  *out = p;
  return FDLBM_OK;
}

void release(fdlbm_handle* h) {
  for (auto& a : h->allocs) {
    if (h->ufree) h->ufree(a.p, a.bytes, h->uctx);
    else cudaFree(a.p);
  }
  h->allocs.clear();
}

// --- geometry -----------------------------------------------------------------------

struct Geo {
  int nx, ny;
  bool px, py;
  std::vector<uint32_t> cls;
  int at(int x, int y) const {
    if (x < 0 || x >= nx) {
      if (!px) return -1;
      x = ((x % nx) + nx) % nx;
    }
    if (y < 0 || y >= ny) {
      if (!py) return -1;
      y = ((y % ny) + ny) % ny;
    }
    return x + nx * y;
  }
  uint32_t cls_at(int x, int y) const {
    int k = at(x, y);
    return k < 0 ? uint32_t(OUTSIDE) : cls[k];
  }
  // Node (x, y) holds a population moving along i: gas, inlet and outlet nodes emit all
  // directions, an interface wall node only towards a gas neighbour.
  bool emits(int x, int y, int i) const {
    uint32_t c = cls_at(x, y);
    if (c == GAS || c == INLET || c == OUTLET) return true;
    return c == WALL && cls_at(x + HEX[i], y + HEY[i]) == GAS;
  }
  uint32_t stencil(int x, int y, int i) const {
    const int ex = HEX[i], ey = HEY[i];
    const bool up2 = emits(x - 2 * ex, y - 2 * ey, i);
    const bool self = emits(x, y, i);
    const bool down = emits(x + ex, y + ey, i);
    const bool up3 = emits(x - 3 * ex, y - 3 * ey, i);
    if (up2 && self) return ST_CENTRAL;
    if (self && down) return ST_FORWARD;
    if (up2 && up3) return ST_BACKWARD;
    if (self) return ST_LIN_S0;
    if (up2) return ST_LIN_S2;
    return ST_NONE;
  }
};

// Unit conversion and the per-species, solid and kinetic parameters shared by the D2Q9
// and D3Q19 handles (Sec. 4.1 units: lattice temperature T / (3 T0), molar masses relative
// to the lightest species, c_j = 1 / sqrt(M_j)). D enters the energy-correction
// coefficient: K_j = (2 c_pj / Pr - (D - 1) / M_j) tau1_j C_j T with c_pj = (D + 2) /
// (2 M_j) (the product-form lattice carries (D - 1) / (D + 2) of the kinetic heat flux).
void set_physics_params(fdlbm_handle* h, const fdlbm_species* species, int ns, const fdlbm_transport* tr,
                        const fdlbm_kinetics* kin, int storage, int D) {
  DevParams& P = h->P;
  double Mmin = 1e300;
  for (int j = 0; j < ns; ++j) Mmin = std::min(Mmin, species[j].M_gmol);
  P.energy_correction = tr->energy_correction ? 1 : 0;
  P.coupling = tr->coupling;
  h->T0 = tr->T0_K;
  const double tl = 1.0 / (3.0 * tr->T0_K);
  const double Tref = tr->T_inlet_K * tl;
  h->T_inlet_lat = Tref;
  h->T_init_lat = tr->T_init_K * tl;
  h->Ts_init_lat = tr->T_solid_init_K * tl;
  // Populations are stored as deviations from the rest equilibrium at T_st, the inlet
  // temperature rounded to a multiple of 2^-12: then the rest factors 1 - T_st, T_st / 2,
  // 1 - 2 T_st and 1 - 3 T_st (1 - T_st) and the rest weights are exact FP32 numbers
  // whose sums over the directions are exactly 1, so that the equilibria formed from
  // them carry no constant rounding bias of mass, momentum or energy.
  const double Tst = std::max(std::round(Tref * 4096.0), 1.0) / 4096.0;
  h->T_st = Tst;
  P.Tref = (float)Tst;
  P.p_out = (float)Tref;  // C_in T_in with C_in = 1
  P.u_inlet = (float)tr->u_inlet;
  P.Tin_lat = (float)Tref;
  P.Tdev_off = (float)(Tst - Tref);
  h->X_init.resize(ns);
  h->X_inlet.resize(ns);
  for (int j = 0; j < ns; ++j) {
    const double M = species[j].M_gmol / Mmin;
    const double c = 1.0 / std::sqrt(M);
    const double t1 = species[j].tau1, t2 = species[j].tau2;
    P.M[j] = (float)M;
    P.invM[j] = (float)(1.0 / M);
    P.sqrtM[j] = (float)std::sqrt(M);
    P.c[j] = (float)c;
    P.sqrtM_lo[j] = (float)(1.0 / double(P.c[j]) - double(P.sqrtM[j]));
    P.c2[j] = (float)(1.0 / M);
    const double a = 1.0 - c;
    P.a[j] = (float)a;
    P.ha[j] = (float)(0.5 * a);
    P.ha2[j] = (float)(0.5 * a * a);
    P.onlattice[j] = (M == 1.0);
    P.rref[j] = (float)(species[j].X_inlet * M);
    P.Xin[j] = (float)species[j].X_inlet;
    P.omega[j] = (float)(2.0 / (1.0 + 2.0 * t1));
    P.t1t2[j] = (float)(t1 / t2);
    P.wt1[j] = (float)(2.0 * t1 / (1.0 + 2.0 * t1));
    P.a2[j] = (float)(1.0 / (2.0 * t2));
    P.inv1a2[j] = (float)(1.0 / (1.0 + 1.0 / (2.0 * t2)));
    P.uc_w[j] = (float)(1.0 / (t2 + 0.5));
    P.invtau2[j] = (float)(1.0 / t2);
    const double cp = (D + 2.0) / (2.0 * M);
    P.kcoef0[j] = tr->energy_correction ? (float)(2.0 * cp / tr->Pr - (D - 1.0) / M) : 0.f;
    P.kcoef[j] = tr->energy_correction ? (float)((2.0 * cp / tr->Pr - (D - 1.0) / M) * t1) : 0.f;
    // Locally updated relaxation times: Wilke's phi_jk (bracket squared, so phi_jj = 1)
    // and 1 / D_jk.
    P.mu_l[j] = (float)species[j].mu;
    for (int q = 0; q < ns; ++q) {
      const double Mq = species[q].M_gmol / Mmin;
      if (tr->local_tau) {
        const double b = 1.0 + std::sqrt(species[j].mu / species[q].mu) * std::pow(Mq / M, 0.25);
        P.phi_w[j][q] = (float)(b * b / std::sqrt(8.0 * (1.0 + M / Mq)));
        P.invD[j][q] = q == j ? 0.f : (float)(1.0 / species[j].D[q]);
      }
    }
    // FP16 storage: deviations |g - rref W0| stay below 2 M_j + rref_j (a population never
    // exceeds its species density, bounded by the molar mass at twice the inlet molar
    // concentration); the largest power of two that maps that bound below 2^15 keeps
    // them inside FP16's range (max 65504) with a factor 2 to spare.
    P.hs[j] = P.hsi[j] = 1.f;
    if (storage == FDLBM_STORAGE_FP16) {
      const double bound = 2.0 * M + species[j].X_inlet * M;
      const int e = (int)std::floor(std::log2(32768.0 / bound));
      P.hs[j] = (float)std::ldexp(1.0, e);
      P.hsi[j] = (float)std::ldexp(1.0, -e);
    }
    h->X_init[j] = species[j].X_init;
    h->X_inlet[j] = species[j].X_inlet;
  }
  P.storage = storage;
  P.local_tau = tr->local_tau ? 1 : 0;
  P.alpha_s = (float)tr->alpha_s;
  P.rhocp_s = (float)tr->rhocp_s;
  P.inv_rhocp_s = (float)(1.0 / tr->rhocp_s);
  P.kappa_f = (float)tr->kappa_f;
  P.dTout = (float)(tr->T_outer_K * tl - Tst);
  P.nr = kin->n_react;
  for (int r = 0; r < kin->n_react; ++r) {
    for (int j = 0; j < ns; ++j) P.nu[r][j] = kin->nu[r][j];
    P.rate_form[r] = kin->rate_form[r];
    P.k0[r] = (float)kin->k0[r];
    P.EaR[r] = (float)(kin->Ea_Jmol[r] / R_GAS);
    P.inv_Keq[r] = kin->rate_form[r] == FDLBM_RATE_XFRAC_REVERSIBLE ? (float)(1.0 / kin->Keq[r]) : 0.f;
    P.heat[r] = (float)(-kin->dH_Jmol[r] / (3.0 * R_GAS * tr->T0_K));
  }
  P.T3T0 = (float)(3.0 * tr->T0_K);
  P.rho_w_tol = (float)kin->rho_w_tol;
  P.rho_w_maxit = kin->rho_w_maxit;
  if (kin->n_react > 0) {
    h->heat0 = -kin->dH_Jmol[0] / (3.0 * R_GAS * tr->T0_K);
    for (int j = 0; j < ns && h->eps_species < 0; ++j)
      if (kin->nu[0][j] < 0) {
        h->eps_species = j;
        h->eps_nu = kin->nu[0][j];
      }
  }
}

fdlbm_status upload_and_init(fdlbm_handle* h, const fdlbm_fields* f);
fdlbm_status create3(const fdlbm_geometry* geom, const fdlbm_species* species, int ns, const fdlbm_transport* tr,
                     const fdlbm_kinetics* kin, const fdlbm_fields* init, const fdlbm_options* opts,
                     fdlbm_handle** out);

}  // namespace

extern "C" {

const char* fdlbm_last_error(void) { return g_err.c_str(); }

fdlbm_status fdlbm_create(const fdlbm_geometry* geom, const fdlbm_species* species, int n_species,
                          const fdlbm_transport* tr, const fdlbm_kinetics* kin, const fdlbm_fields* init,
                          const fdlbm_options* opts, fdlbm_handle** out) {
  if (!out) return fail(FDLBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!geom || !species || !tr || !kin || !geom->mask)
    return fail(FDLBM_EINVAL, "geometry, species, transport, kinetics and mask are required");
  if (geom->lattice != FDLBM_D2Q9 && geom->lattice != FDLBM_D3Q19)
    return fail(FDLBM_EINVAL, "lattice must be FDLBM_D2Q9 or FDLBM_D3Q19 (got %d)", geom->lattice);
  if (geom->nx < 4 || geom->ny < 4) return fail(FDLBM_EINVAL, "lattice must be at least 4x4 (got %dx%d)", geom->nx, geom->ny);
  if ((long long)geom->nx * geom->ny > (1LL << 29)) return fail(FDLBM_EINVAL, "lattice too large (at most 2^29 nodes)");
  if (n_species < 1 || n_species > MAX_NS) return fail(FDLBM_EINVAL, "n_species must be 1..%d", MAX_NS);
  if (kin->n_react < 0 || kin->n_react > MAX_NR) return fail(FDLBM_EINVAL, "n_react must be 0..%d", MAX_NR);
  const int* fb = geom->face_bc;
  for (int f = 0; f < 4; ++f)
    if (fb[f] < 0 || fb[f] > 4) return fail(FDLBM_EINVAL, "face_bc[%d] invalid", f);
  if ((fb[0] == FDLBM_FACE_PERIODIC) != (fb[1] == FDLBM_FACE_PERIODIC) ||
      (fb[2] == FDLBM_FACE_PERIODIC) != (fb[3] == FDLBM_FACE_PERIODIC))
    return fail(FDLBM_EINVAL, "periodic faces must come in pairs");
  if (fb[1] == FDLBM_FACE_INLET || fb[0] == FDLBM_FACE_OUTLET || fb[2] == FDLBM_FACE_INLET ||
      fb[3] == FDLBM_FACE_INLET || fb[2] == FDLBM_FACE_OUTLET || fb[3] == FDLBM_FACE_OUTLET)
    return fail(FDLBM_EINVAL, "inlet only on x-, outlet only on x+");
  {
    // A node writes the periodic copy for one face only, so no node may lie within the
    // ghost depth of both faces of a periodic axis.
    const int minp = 2 * (geom->lattice == FDLBM_D3Q19 ? GHOST3 : GHOST);
    const int len[3] = {geom->nx, geom->ny, geom->lattice == FDLBM_D3Q19 ? geom->nz : minp};
    for (int a = 0; a < (geom->lattice == FDLBM_D3Q19 ? 3 : 2); ++a)
      if (fb[2 * a] == FDLBM_FACE_PERIODIC && len[a] < minp)
        return fail(FDLBM_EINVAL, "periodic axis %d has %d nodes; at least %d are needed", a, len[a], minp);
  }
  if (!(tr->T0_K > 0) || !(tr->T_inlet_K > 0) || !(tr->T_init_K > 0) || !(tr->T_solid_init_K > 0))
    return fail(FDLBM_EINVAL, "temperatures must be positive");
  if (!(tr->Pr > 0)) return fail(FDLBM_EINVAL, "Pr must be positive");
  if (tr->alpha_s < 0 || tr->alpha_s > 0.25 || !(tr->rhocp_s > 0))
    return fail(FDLBM_EINVAL, "alpha_s must be in [0, 1/4] (explicit FD stability in 2D) and rhocp_s > 0");
  if (tr->coupling != FDLBM_COUPLING_CONSERVATIVE && tr->coupling != FDLBM_COUPLING_PAPER)
    return fail(FDLBM_EINVAL, "unknown coupling");
  if (kin->rho_w_maxit < 1 || !(kin->rho_w_tol > 0)) return fail(FDLBM_EINVAL, "rho_w_tol > 0 and rho_w_maxit >= 1 required");
  const int storage = opts ? opts->storage : FDLBM_STORAGE_FP32;
  if (storage != FDLBM_STORAGE_FP32 && storage != FDLBM_STORAGE_BF16 && storage != FDLBM_STORAGE_FP16)
    return fail(FDLBM_EINVAL, "unsupported storage %d", storage);

  for (int j = 0; j < n_species; ++j)
    if (!(species[j].M_gmol > 0) || !(species[j].tau1 > 0) || !(species[j].tau2 > 0))
      return fail(FDLBM_EINVAL, "species %d: M, tau1, tau2 must be positive", j);
  for (int r = 0; r < kin->n_react; ++r) {
    if (kin->rate_form[r] != FDLBM_RATE_CONC_BILINEAR && kin->rate_form[r] != FDLBM_RATE_XFRAC_REVERSIBLE)
      return fail(FDLBM_EINVAL, "reaction %d: unknown rate form", r);
    if (kin->rate_form[r] == FDLBM_RATE_XFRAC_REVERSIBLE && !(kin->Keq[r] > 0))
      return fail(FDLBM_EINVAL, "reaction %d: Keq must be positive", r);
    for (int j = 0; j < n_species; ++j)
      if (kin->nu[r][j] < -4 || kin->nu[r][j] > 4) return fail(FDLBM_EINVAL, "reaction %d: |nu| <= 4", r);
  }

  if (tr->local_tau) {
    if (geom->lattice != FDLBM_D2Q9) return fail(FDLBM_EINVAL, "local relaxation times are implemented for D2Q9");
    if (storage != FDLBM_STORAGE_FP32) return fail(FDLBM_EINVAL, "local relaxation times need FP32 storage");
    if (n_species < 2) return fail(FDLBM_EINVAL, "local relaxation times need at least 2 species");
    for (int j = 0; j < n_species; ++j) {
      if (!(species[j].mu > 0)) return fail(FDLBM_EINVAL, "species %d: mu must be positive", j);
      for (int k = 0; k < n_species; ++k)
        if (k != j && !(species[j].D[k] > 0)) return fail(FDLBM_EINVAL, "species %d: D[%d] must be positive", j, k);
    }
  }
  if (opts && opts->ledger_detail && (storage != FDLBM_STORAGE_FP32 || tr->local_tau))
    return fail(FDLBM_EINVAL, "exact accounts need FP32 storage and constant relaxation times");
  if (opts && (opts->tile_entries != 0 && (opts->tile_entries % 32 != 0 || opts->tile_entries < 64 ||
                                           opts->tile_entries > STEP_BLOCK)))
    return fail(FDLBM_EINVAL, "tile_entries must be 0 or a multiple of 32 in [64, %d] (got %d)", STEP_BLOCK,
                opts->tile_entries);
  if (opts && opts->wall_order != 0 && opts->wall_order != 1)
    return fail(FDLBM_EINVAL, "wall_order must be 0 or 1 (got %d)", opts->wall_order);
  {
    // Mole fractions: each in [0, 1], summing to 1 (initial and inlet composition).
    double sx0 = 0.0, sx1 = 0.0;
    for (int j = 0; j < n_species; ++j) {
      if (!(species[j].X_init >= 0 && species[j].X_init <= 1) || !(species[j].X_inlet >= 0 && species[j].X_inlet <= 1))
        return fail(FDLBM_EINVAL, "species %d: mole fractions must lie in [0, 1]", j);
      sx0 += species[j].X_init;
      sx1 += species[j].X_inlet;
    }
    if (std::fabs(sx0 - 1.0) > 1e-6 || std::fabs(sx1 - 1.0) > 1e-6)
      return fail(FDLBM_EINVAL, "mole fractions must sum to 1 (initial %.9g, inlet %.9g)", sx0, sx1);
    // The product-form equilibrium (Eq. eq_state_pop) needs a positive rest factor
    // 1 - M_j u^2 - T for every species (M_j relative to the lightest species, T in
    // lattice units T_K / (3 T0)).
    double Mmin = species[0].M_gmol, Mmax = species[0].M_gmol;
    for (int j = 1; j < n_species; ++j) {
      Mmin = std::min(Mmin, species[j].M_gmol);
      Mmax = std::max(Mmax, species[j].M_gmol);
    }
    const double Mr = Mmax / Mmin, u = tr->u_inlet;
    const double Tin = tr->T_inlet_K / (3.0 * tr->T0_K), T0 = tr->T_init_K / (3.0 * tr->T0_K);
    if (!(Mr * u * u + Tin < 1.0))
      return fail(FDLBM_EINVAL, "inlet state outside the equilibrium's range: 1 - M u^2 - T = %.6g <= 0 "
                  "(T_lat %.6g, u %.6g, heaviest M %.6g)", 1.0 - Mr * u * u - Tin, Tin, u, Mr);
    if (!(T0 < 1.0)) return fail(FDLBM_EINVAL, "initial temperature outside the equilibrium's range: T_lat %.6g >= 1", T0);
  }
  if (geom->lattice == FDLBM_D3Q19) return create3(geom, species, n_species, tr, kin, init, opts, out);

  fdlbm_handle* h = new fdlbm_handle();
  h->device = opts ? opts->device : 0;
  DeviceGuard guard(h->device);
  h->stream = opts ? (cudaStream_t)opts->stream : nullptr;
  if (opts) {
    h->ualloc = opts->alloc;
    h->ufree = opts->free;
    h->uctx = opts->alloc_ctx;
  }
  const int nx = geom->nx, ny = geom->ny, n = nx * ny, ns = n_species;
  h->nx = nx;
  h->ny = ny;
  h->ns = ns;

  // Node classes.
  Geo G;
  G.nx = nx;
  G.ny = ny;
  G.px = fb[0] == FDLBM_FACE_PERIODIC;
  G.py = fb[2] == FDLBM_FACE_PERIODIC;
  G.cls.assign(n, GAS);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int k = x + nx * y;
      const uint8_t m = geom->mask[k];
      if (m > 2) {
        delete h;
        return fail(FDLBM_EINVAL, "mask value %d at (%d,%d)", m, x, y);
      }
      if (m == FDLBM_MASK_GAS) {
        if (x == 0 && fb[0] == FDLBM_FACE_INLET) G.cls[k] = INLET;
        else if (x == nx - 1 && fb[1] == FDLBM_FACE_OUTLET) G.cls[k] = OUTLET;
        else G.cls[k] = GAS;
      } else {
        G.cls[k] = SOLID;
      }
    }
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int k = x + nx * y;
      if (G.cls[k] != SOLID) continue;
      for (int i = 1; i < Q; ++i)
        if (G.cls_at(x + HEX[i], y + HEY[i]) == GAS) G.cls[k] = WALL;
    }
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int k = x + nx * y;
      if (G.cls[k] == GAS) {
        for (int i = 1; i < Q; ++i)
          if (G.at(x + HEX[i], y + HEY[i]) < 0) {
            delete h;
            return fail(FDLBM_EGEOM, "gas node (%d,%d) touches a closed lattice face", x, y);
          }
      } else if (G.cls[k] == OUTLET && G.cls[k - 1] != GAS) {
        delete h;
        return fail(FDLBM_EGEOM, "outlet node (%d,%d) has no upstream gas node", x, y);
      }
    }
  // Code words: class, catalytic bit, per-direction stencils (gas: every direction;
  // wall: arrival directions, others marked NOT_ARRIVAL).
  h->code.assign(n, 0);
  std::vector<int32_t> walls, solids;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int k = x + nx * y;
      const uint32_t c = G.cls[k];
      uint32_t w = c;
      if (geom->mask[k] == FDLBM_MASK_CATALYTIC) w |= CATALYTIC_BIT;
      if (c == GAS) {
        for (int i = 1; i < Q; ++i) {
          const uint32_t st = G.stencil(x, y, i);
          w |= st << (STENCIL_SHIFT + 3 * (i - 1));
          h->stencil_counts[st]++;
        }
      } else if (c == WALL) {
        for (int i = 1; i < Q; ++i) {
          uint32_t st = ST_NOT_ARRIVAL;
          if (G.cls_at(x - HEX[i], y - HEY[i]) == GAS) {
            st = G.stencil(x, y, i);
            h->stencil_counts[st]++;
          }
          w |= st << (STENCIL_SHIFT + 3 * (i - 1));
        }
        walls.push_back(k);
      } else if (c == SOLID) {
        solids.push_back(k);
      }
      // Bits 28..31: gas nodes flag gas neighbours, solid nodes flag solid neighbours,
      // along directions 1..4.
      if (c == GAS)
        for (int i = 1; i <= 4; ++i)
          if (G.cls_at(x + HEX[i], y + HEY[i]) == GAS) w |= 1u << (NBR_GAS_SHIFT + i - 1);
      if (c == WALL || c == SOLID)
        for (int i = 1; i <= 4; ++i) {
          const uint32_t cn = G.cls_at(x + HEX[i], y + HEY[i]);
          if (cn == WALL || cn == SOLID) w |= 1u << (NBR_GAS_SHIFT + i - 1);
        }
      h->code[k] = w;
      h->counts[c]++;
    }
  if (opts && opts->strict_geometry) {
    // Reading R6: the linear and no-interpolation fallbacks serve concave corners and one-
    // or two-node gaps, which the paper's geometries exclude.
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const uint32_t w = h->code[x + nx * y], c = node_class(w);
        if (c != GAS && c != WALL) continue;
        for (int i = 1; i < Q; ++i) {
          const uint32_t st = stencil_of(w, i);
          if (st == ST_NONE || st == ST_LIN_S0 || st == ST_LIN_S2) {
            delete h;
            return fail(FDLBM_EGEOM, "strict geometry: %s node (%d,%d) pulls direction %d without a quadratic "
                        "stencil (concave corner or narrow gap)", c == GAS ? "gas" : "wall", x, y, i);
          }
        }
      }
  }
  std::vector<int32_t> solid_list(walls);
  solid_list.insert(solid_list.end(), solids.begin(), solids.end());

  // Parameters (Sec. 4.1 units).
  DevParams& P = h->P;
  P.nx = nx;
  P.ny = ny;
  P.n = n;
  P.xoff = XOFF;
  P.yoff = YOFF;
  P.pitch = (nx + XOFF + 2 * GHOST + 31) / 32 * 32;
  P.plane = ((long long)P.pitch * (ny + 2 * YOFF) + 63) / 64 * 64;
  // Kernels address populations with 32-bit element offsets.
  if ((long long)ns * Q * P.plane >= (1LL << 31)) {
    const long long plane = P.plane;  // P refers into h
    delete h;
    return fail(FDLBM_EINVAL, "lattice too large: %d species x 9 x %lld padded cells exceed 2^31 elements",
                ns, plane);
  }
  std::vector<int2> gas_list;
  gas_list.reserve((size_t)h->counts[GAS]);
  // Code words on the padded lattice: ghost cells within GHOST of a periodic face carry
  // the wrapped node's word, everything else outside the lattice is OUTSIDE.
  std::vector<uint32_t> pcode((size_t)P.plane, uint32_t(OUTSIDE));
  for (int py = 0; py < ny + 2 * YOFF; ++py)
    for (int px = 0; px < P.pitch; ++px) {
      int x = px - XOFF, y = py - YOFF;
      if (x < 0 || x >= nx) {
        if (!G.px || x < -GHOST || x >= nx + GHOST) continue;
        x = x < 0 ? x + nx : x - nx;
      }
      if (y < 0 || y >= ny) {
        if (!G.py || y < -GHOST || y >= ny + GHOST) continue;
        y = y < 0 ? y + ny : y - ny;
      }
      pcode[(size_t)px + (size_t)py * P.pitch] = h->code[x + nx * y];
    }
  // Gas tiles and step-kernel blocks. Rows are taken in bands of `band` rows; each band
  // is split along x into column ranges whose gas nodes (the tile's interior) plus the
  // gas nodes of the one-node ring around it that neighbour them along an axis (its
  // halo, needed for the energy-correction divergence at the current time level) fit
  // one block, and whose moment map ((columns + 2) x (rows + 2) slots) fits
  // GAS_MAP_SLOTS. Ring positions wrap on periodic axes (a range spanning a whole
  // periodic axis repeats nodes of its own interior in the ring). Without the energy
  // correction tiles have no halo. Blocks of a band: its gas tiles, then its wall
  // blocks; the interior solid blocks come last.
  const bool phi = tr->energy_correction != 0;
  std::vector<int4> blocks;
  std::vector<uint16_t> gas_slot;
  {
    const int band = std::min(64, (opts && opts->band_rows > 0) ? opts->band_rows : 16);
    const int cap = (opts && opts->tile_entries > 0) ? opts->tile_entries : STEP_BLOCK;
    const bool walls_last = opts && opts->wall_order == 1;
    P.block_threads = cap;
    auto is_gas = [&](int x, int y) { return G.cls_at(x, y) == GAS; };
    std::vector<int> wall_row(ny + 1, 0);
    for (int y = 0, w = 0; y <= ny; ++y) {
      wall_row[y] = w;
      if (y == ny) break;
      for (int x = 0; x < nx; ++x) w += G.cls[x + nx * y] == WALL;
    }
    // The wall nodes of a band, sorted by their set of arrival directions (stable, so by
    // position within a set): the lanes of a warp then share their arrival and emission
    // directions, and a warp steps through the union of its lanes' directions (on the
    // 1024x512 bed with bands of 8 rows: 3.6 directions on average instead of 8.0 in
    // row-major order; 2.6 per node).
    {
      auto arrivals = [&](int32_t k) {
        uint32_t m = 0;
        for (int i = 1; i < Q; ++i)
          if (stencil_of(h->code[k], i) != ST_NOT_ARRIVAL) m |= 1u << i;
        return m;
      };
      for (int y0 = 0; y0 < ny; y0 += band) {
        const int y1 = std::min(ny, y0 + band);
        std::stable_sort(walls.begin() + wall_row[y0], walls.begin() + wall_row[y1],
                         [&](int32_t a, int32_t b) { return arrivals(a) < arrivals(b); });
      }
      std::copy(walls.begin(), walls.end(), solid_list.begin());
    }
    auto chunks = [&](int first, int last) {
      for (int s0 = first; s0 < last; s0 += cap) blocks.push_back(make_int4(1, s0, std::min(cap, last - s0), 0));
    };
    auto push_entry = [&](int x, int y, int aux, int slot) {
      const int wx = ((x % nx) + nx) % nx, wy = ((y % ny) + ny) % ny;
      gas_list.push_back(make_int2((wx + XOFF) + (wy + YOFF) * P.pitch, aux));
      gas_slot.push_back((uint16_t)slot);
    };
    std::vector<int> col_int(nx), col_tb(nx);
    for (int y0 = 0; y0 < ny; y0 += band) {
      const int y1 = std::min(ny, y0 + band), H = y1 - y0;
      // per column: interior gas nodes, and top/bottom ring nodes it needs
      for (int x = 0; x < nx; ++x) {
        int c = 0;
        for (int y = y0; y < y1; ++y) c += is_gas(x, y);
        col_int[x] = c;
        col_tb[x] = phi ? int(is_gas(x, y0 - 1) && is_gas(x, y0)) + int(is_gas(x, y1) && is_gas(x, y1 - 1)) : 0;
      }
      auto side = [&](int xs, int xin) {  // ring column xs beside interior column xin
        if (!phi) return 0;
        int c = 0;
        for (int y = y0; y < y1; ++y) c += is_gas(xs, y) && is_gas(xin, y);
        return c;
      };
      for (int x0 = 0; x0 < nx;) {
        const int left = side(x0 - 1, x0);
        int x1 = x0 + 1, inner = col_int[x0] + col_tb[x0];
        while (x1 < nx) {
          const int more = inner + col_int[x1] + col_tb[x1];
          if (left + more + side(x1 + 1, x1) > cap) break;
          if (phi && (x1 + 1 - x0 + 2) * (H + 2) > GAS_MAP_SLOTS) break;
          inner = more;
          ++x1;
        }
        const int W = x1 - x0, Wp = W + 2;
        const int first = (int)gas_list.size();
        for (int y = y0; y < y1; ++y)
          for (int x = x0; x < x1; ++x)
            if (G.cls[x + nx * y] == GAS) {
              const bool near_x = G.px && (x < GHOST || x >= nx - GHOST);
              const bool near_y = G.py && (y < GHOST || y >= ny - GHOST);
              const bool outlet = x + 1 == nx - 1 && G.cls[x + 1 + nx * y] == OUTLET;
              const int aux = (x + nx * y) | (outlet ? GAS_AUX_OUTLET : 0) | (near_x || near_y ? GAS_AUX_GHOST : 0);
              push_entry(x, y, aux, phi ? (x - x0 + 1) + (y - y0 + 1) * Wp : 0);
            }
        const int n_int = (int)gas_list.size() - first;
        if (phi) {
          for (int x = x0; x < x1; ++x) {
            if (is_gas(x, y0 - 1) && is_gas(x, y0)) push_entry(x, y0 - 1, 0, x - x0 + 1);
            if (is_gas(x, y1) && is_gas(x, y1 - 1)) push_entry(x, y1, 0, (x - x0 + 1) + (H + 1) * Wp);
          }
          for (int y = y0; y < y1; ++y) {
            if (is_gas(x0 - 1, y) && is_gas(x0, y)) push_entry(x0 - 1, y, 0, (y - y0 + 1) * Wp);
            if (is_gas(x1, y) && is_gas(x1 - 1, y)) push_entry(x1, y, 0, (W + 1) + (y - y0 + 1) * Wp);
          }
        }
        const int n_tot = (int)gas_list.size() - first;
        if (n_int > 0) blocks.push_back(make_int4(0, first, (n_int << 16) | n_tot, Wp));
        else {
          gas_list.resize(first);
          gas_slot.resize(first);
        }
        x0 = x1;
      }
      if (!walls_last) chunks(wall_row[y0], wall_row[y1]);
    }
    if (walls_last) chunks(0, (int)walls.size());
    chunks((int)walls.size(), (int)solid_list.size());
  }
  P.n_gas = h->counts[GAS];
  P.n_blocks = (int)blocks.size();
  h->blocks_host = blocks;
  P.ns = ns;
  P.periodic_x = G.px;
  P.periodic_y = G.py;
  P.n_solid_list = (int)solid_list.size();
  P.n_wall_list = (int)walls.size();
  for (int f = 0; f < 4; ++f) P.fixedT_face[f] = fb[f] == FDLBM_FACE_FIXED_T;
  set_physics_params(h, species, ns, tr, kin, storage, 2);
  P.ledger_detail = (opts && opts->ledger_detail) ? 1 : 0;
  const double Tref = h->T_st;
  for (int i = 0; i < Q; ++i) {
    const double wx = HEX[i] == 0 ? 1.0 - Tref : 0.5 * Tref;
    const double wy = HEY[i] == 0 ? 1.0 - Tref : 0.5 * Tref;
    P.W0[i] = (float)(wx * wy);
  }
  // Inlet velocity per row: plug, or a parabola vanishing on the bounding wall nodes of
  // each contiguous inlet run.
  h->inlet_u.assign(ny, 0.0);
  for (int y = 0; y < ny; ++y) {
    if (G.cls[0 + nx * y] != INLET) continue;
    if (tr->inlet_profile == FDLBM_PROFILE_PLUG) {
      h->inlet_u[y] = tr->u_inlet;
      continue;
    }
    int y0 = y, y1 = y;
    while (y0 - 1 >= 0 && G.cls[nx * (y0 - 1)] == INLET) --y0;
    while (y1 + 1 < ny && G.cls[nx * (y1 + 1)] == INLET) ++y1;
    const double H = double(y1 - y0 + 2), s = double(y - y0 + 1) / H;
    h->inlet_u[y] = 4.0 * tr->u_inlet * s * (1.0 - s);
  }

  // Device state.
  fdlbm_status st;
  DevState& S = h->S;
  const size_t pop_bytes = pop_bytes_per_value(storage) * (size_t)ns * Q * (size_t)P.plane;
  void* p;
  for (int b = 0; b < 2; ++b) {
    if ((st = dalloc(h, pop_bytes, &p)) != FDLBM_OK) { release(h); delete h; return st; }
    S.h[b] = p;
    if ((st = dalloc(h, sizeof(float) * n, &p)) != FDLBM_OK) { release(h); delete h; return st; }
    S.Ts[b] = (float*)p;
  }
#define ALLOC(field, type, count)                                                    \
  if ((st = dalloc(h, sizeof(type) * (size_t)(count), &p)) != FDLBM_OK) {             \
    release(h);                                                                      \
    delete h;                                                                        \
    return st;                                                                       \
  }                                                                                  \
  field = (type*)p;
  ALLOC(S.code, uint32_t, P.plane);
  ALLOC(S.solid_list, int32_t, std::max<size_t>(solid_list.size(), 1));
  ALLOC(S.gas_list, int2, std::max<size_t>(gas_list.size(), 1));
  ALLOC(S.gas_slot, uint16_t, std::max<size_t>(gas_slot.size(), 1));
  ALLOC(S.blocks, int4, std::max<size_t>(blocks.size(), 1));
  ALLOC(S.mom, float, (size_t)(ns + 3) * n);
  ALLOC(S.Tgas, float, 2 * (size_t)n);
  ALLOC(S.snap, float, (size_t)(ns + 4) * n);
  ALLOC(S.ledger, double, (size_t)LG_COUNT * ledger_slots(P));
  ALLOC(S.rw, float, (size_t)ns * std::max<size_t>(walls.size(), 1));
  ALLOC(S.flags, int, 4);
  ALLOC(S.red, double, totals_count(ns) + residual_count3(ns) + LG_COUNT + 8);
  ALLOC(h->out_buf, float, (size_t)(2 * ns + 4) * n);
  std::vector<float2> wall_u;
  if (geom->wall_u) {
    // velocity of every wall-list entry (moving diffusive walls)
    wall_u.resize(std::max<size_t>(walls.size(), 1), make_float2(0.f, 0.f));
    for (size_t q = 0; q < walls.size(); ++q)
      wall_u[q] = make_float2((float)geom->wall_u[walls[q]], (float)geom->wall_u[(size_t)n + walls[q]]);
    ALLOC(S.wall_u, float2, wall_u.size());
  }
#undef ALLOC
  cudaError_t e = cudaMemcpyAsync(S.code, pcode.data(), sizeof(uint32_t) * pcode.size(), cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess && !solid_list.empty())
    e = cudaMemcpyAsync(S.solid_list, solid_list.data(), sizeof(int32_t) * solid_list.size(),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && !blocks.empty())
    e = cudaMemcpyAsync(S.blocks, blocks.data(), sizeof(int4) * blocks.size(), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && !gas_list.empty())
    e = cudaMemcpyAsync(S.gas_list, gas_list.data(), sizeof(int2) * gas_list.size(), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess && !gas_slot.empty())
    e = cudaMemcpyAsync(S.gas_slot, gas_slot.data(), sizeof(uint16_t) * gas_slot.size(), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess && !wall_u.empty())
    e = cudaMemcpyAsync(S.wall_u, wall_u.data(), sizeof(float2) * wall_u.size(), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    release(h);
    delete h;
    return cuda_fail(e, "upload geometry");
  }
  if ((st = upload_and_init(h, init)) != FDLBM_OK) {
    release(h);
    delete h;
    return st;
  }
  *out = h;
  return FDLBM_OK;
}

fdlbm_status fdlbm_step(fdlbm_handle* h, int64_t n) {
  if (!h || n < 0) return fail(FDLBM_EINVAL, "bad handle or step count");
  DeviceGuard guard(h->device);
  for (int64_t k = 0; k < n; ++k) {
    if (h->profiling && h->events_used + 2 <= h->events.size()) {
      cudaEvent_t* ev = h->events.data() + h->events_used;
      CK(cudaEventRecord(ev[0], h->stream), "event record");
      if (h->dim == 3) CK(launch_step3(h->P, h->S, h->cur, false, h->stream, uint32_t(h->steps + k)), "step launch");
      else CK(launch_step(h->P, h->S, h->cur, false, h->stream, uint32_t(h->steps + k)), "step launch");
      CK(cudaEventRecord(ev[1], h->stream), "event record");
      h->events_used += 2;
    } else if (h->dim == 3) {
      CK(launch_step3(h->P, h->S, h->cur, false, h->stream, uint32_t(h->steps + k)), "step launch");
    } else {
      CK(launch_step(h->P, h->S, h->cur, false, h->stream, uint32_t(h->steps + k)), "step launch");
    }
    h->cur ^= 1;
  }
  if (n > 0) h->mom_fresh = false;
  h->steps += n;
  return FDLBM_OK;
}

fdlbm_status fdlbm_sync(fdlbm_handle* h) {
  if (!h) return fail(FDLBM_EINVAL, "bad handle");
  DeviceGuard guard(h->device);
  int flags = 0;
  CK(cudaMemcpyAsync(&flags, h->S.flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read flags");
  CK(cudaStreamSynchronize(h->stream), "stream sync");
  if (flags) return fail(FDLBM_EUNSTABLE, "non-finite or non-positive density/temperature seen in the gas");
  return FDLBM_OK;
}

}  // extern "C"

namespace {

fdlbm_status ensure_moments(fdlbm_handle* h) {
  if (h->mom_fresh) return FDLBM_OK;
  // The buffer read by the last step still holds its input: recompute that step's
  // pre-collision moments (time t) from it.
  if (h->dim == 3) CK(launch_step3(h->P, h->S, h->cur ^ 1, true, h->stream), "moments launch");
  else CK(launch_step(h->P, h->S, h->cur ^ 1, true, h->stream), "moments launch");
  h->mom_fresh = true;
  return FDLBM_OK;
}

fdlbm_status read_totals(fdlbm_handle* h, double* tot) {
  fdlbm_status st = ensure_moments(h);
  if (st != FDLBM_OK) return st;
  if (h->dim == 3) CK(launch_totals3(h->P, h->S, h->cur, h->stream), "totals launch");
  else CK(launch_totals(h->P, h->S, h->cur, h->stream), "totals launch");
  CK(cudaMemcpyAsync(tot, h->S.red, sizeof(double) * totals_count(h->ns), cudaMemcpyDeviceToHost, h->stream),
     "read totals");
  CK(cudaStreamSynchronize(h->stream), "stream sync");
  return FDLBM_OK;
}

// Energy of the stored populations (exact accounts), into *out.
fdlbm_status read_pop_energy(fdlbm_handle* h, double* out) {
  double* slot = h->S.red + totals_count(h->ns) + residual_count3(h->ns) + LG_COUNT;
  CK(launch_pop_energy(h->P, h->S, h->cur, slot, h->stream), "population energy");
  CK(cudaMemcpyAsync(out, slot, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "read population energy");
  CK(cudaStreamSynchronize(h->stream), "stream sync");
  return FDLBM_OK;
}

fdlbm_status upload_and_init3(fdlbm_handle* h, const fdlbm_fields* f);

// Initial fields the equilibrium can represent: mole fractions summing to 1 (a trace
// species may sit slightly below zero, as the solver's own fields can after the
// interpolation's undershoot), and a positive rest factor 1 - M_j u_a^2 - T on every axis
// for the heaviest species (Eq. eq_state_pop; T and u in lattice units).
fdlbm_status check_initial_state(const fdlbm_handle* h, const std::vector<double>& X, const std::vector<double>& u,
                                 const std::vector<double>& T, long n, int dim) {
  float Mmax = 0.f;
  for (int j = 0; j < h->ns; ++j) Mmax = std::max(Mmax, h->P.M[j]);
  for (long k = 0; k < n; ++k) {
    double sx = 0.0;
    for (int j = 0; j < h->ns; ++j) {
      const double x = X[(size_t)j * n + k];
      if (!(x >= -1e-3)) return fail(FDLBM_EINVAL, "initial mole fraction %d at node %ld is negative (%.3g)", j, k, x);
      sx += x;
    }
    if (std::fabs(sx - 1.0) > 1e-6) return fail(FDLBM_EINVAL, "initial mole fractions at node %ld sum to %.9g", k, sx);
    for (int a = 0; a < dim; ++a) {
      const double ua = u[(size_t)a * n + k];
      if (!(1.0 - double(Mmax) * ua * ua - T[k] > 0.0))
        return fail(FDLBM_EINVAL, "initial state at node %ld outside the equilibrium's range: "
                    "1 - M u^2 - T = %.6g <= 0", k, 1.0 - double(Mmax) * ua * ua - T[k]);
    }
  }
  return FDLBM_OK;
}

fdlbm_status upload_and_init(fdlbm_handle* h, const fdlbm_fields* f) {
  if (h->dim == 3) return upload_and_init3(h, f);
  const int n = h->nx * h->ny, ns = h->ns;
  const double tl = 1.0 / (3.0 * h->T0);
  std::vector<double> X((size_t)ns * n), u(2 * (size_t)n, 0.0), T(n), Ts(n), C(n, 1.0);
  for (int j = 0; j < ns; ++j)
    for (int k = 0; k < n; ++k) X[(size_t)j * n + k] = (f && f->X) ? f->X[(size_t)j * n + k] : h->X_init[j];
  if (f && f->u) std::memcpy(u.data(), f->u, sizeof(double) * 2 * n);
  for (int k = 0; k < n; ++k) {
    T[k] = (f && f->T_K) ? f->T_K[k] * tl : h->T_init_lat;
    Ts[k] = (f && f->Ts_K) ? f->Ts_K[k] * tl : h->Ts_init_lat;
    if (f && f->C) C[k] = f->C[k];
    if (!(T[k] > 0) || !(C[k] > 0)) return fail(FDLBM_EINVAL, "initial T and C must be positive (node %d)", k);
  }
  if (fdlbm_status st = check_initial_state(h, X, u, T, n, 2); st != FDLBM_OK) return st;
  std::vector<double> inlet(h->inlet_u);
  inlet.insert(inlet.end(), h->X_inlet.begin(), h->X_inlet.end());
  inlet.push_back(h->T_inlet_lat);
  // Temporary device copies of the FP64 fields.
  const size_t total = X.size() + u.size() + T.size() + Ts.size() + C.size() + inlet.size();
  double* d = nullptr;
  CK(cudaMalloc(&d, sizeof(double) * total), "init staging alloc");
  size_t off = 0;
  double* dX = d + off; off += X.size();
  double* du = d + off; off += u.size();
  double* dT = d + off; off += T.size();
  double* dTs = d + off; off += Ts.size();
  double* dC = d + off; off += C.size();
  double* dIn = d + off;
  cudaError_t e = cudaSuccess;
  auto up = [&](double* dst, const std::vector<double>& v) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, h->stream);
  };
  up(dX, X);
  up(du, u);
  up(dT, T);
  up(dTs, Ts);
  up(dC, C);
  up(dIn, inlet);
  if (e == cudaSuccess) e = launch_init(h->P, h->S, dX, du, dT, dTs, dC, dIn, h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->S.ledger, 0, sizeof(double) * LG_COUNT * ledger_slots(h->P), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->S.flags, 0, sizeof(int) * 4, h->stream);
  // no previous wall densities yet: all-ones bytes are a NaN
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->S.rw, 0xFF, sizeof(float) * (size_t)ns * std::max(h->P.n_wall_list, 1), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "initialise state");
  h->cur = 0;
  h->steps = 0;
  h->steps_at_residual = 0;
  h->have_snap = false;
  h->mom_fresh = true;
  std::vector<double> tot(totals_count(ns));
  fdlbm_status st = read_totals(h, tot.data());
  if (st != FDLBM_OK) return st;
  h->E0 = tot[0];
  h->H0 = tot[1];
  for (int j = 0; j < ns; ++j) {
    h->mass0[j] = tot[2 + j];
    h->moles0[j] = tot[2 + ns + j];
  }
  h->E_pop0 = 0.0;
  if (h->P.ledger_detail) {
    st = read_pop_energy(h, &h->E_pop0);
    if (st != FDLBM_OK) return st;
  }
  return FDLBM_OK;
}


// ---- D3Q19 handles ------------------------------------------------------------------
// D3Q19 velocities in the order of the 3D kernels (rest, +-x, +-y, +-z, face diagonals).
constexpr int H3X[Q19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int H3Y[Q19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
constexpr int H3Z[Q19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

struct Geo3 {
  int nx, ny, nz;
  bool px, py, pz;
  std::vector<uint32_t> cls;
  static int wrap(int v, int len, bool per) {
    if (v >= 0 && v < len) return v;
    return per ? ((v % len) + len) % len : -1;
  }
  long at(int x, int y, int z) const {
    x = wrap(x, nx, px);
    y = wrap(y, ny, py);
    z = wrap(z, nz, pz);
    if (x < 0 || y < 0 || z < 0) return -1;
    return x + (long)nx * (y + (long)ny * z);
  }
  uint32_t cls_at(int x, int y, int z) const {
    const long k = at(x, y, z);
    return k < 0 ? uint32_t(OUTSIDE) : cls[k];
  }
  // Node (x, y, z) holds a population moving along i (reading R6).
  bool emits(int x, int y, int z, int i) const {
    const uint32_t c = cls_at(x, y, z);
    if (c == GAS || c == INLET || c == OUTLET) return true;
    return c == WALL && cls_at(x + H3X[i], y + H3Y[i], z + H3Z[i]) == GAS;
  }
  uint32_t stencil(int x, int y, int z, int i) const {
    const int ex = H3X[i], ey = H3Y[i], ez = H3Z[i];
    const bool up2 = emits(x - 2 * ex, y - 2 * ey, z - 2 * ez, i);
    const bool self = emits(x, y, z, i);
    const bool down = emits(x + ex, y + ey, z + ez, i);
    const bool up3 = emits(x - 3 * ex, y - 3 * ey, z - 3 * ez, i);
    if (up2 && self) return ST_CENTRAL;
    if (self && down) return ST_FORWARD;
    if (up2 && up3) return ST_BACKWARD;
    if (self) return ST_LIN_S0;
    if (up2) return ST_LIN_S2;
    return ST_NONE;
  }
};

// D3Q19 rest-equilibrium weight of direction i at lattice temperature T.
double wrest3_h(int i, double T) {
  const int nz = (H3X[i] != 0) + (H3Y[i] != 0) + (H3Z[i] != 0);
  if (nz == 0) return (1.0 - T) * (1.0 - T) * (1.0 - T) + T * T * T;
  if (nz == 1) return 0.5 * T * (1.0 - 2.0 * T);
  return 0.25 * T * T;
}

fdlbm_status create3(const fdlbm_geometry* geom, const fdlbm_species* species, int ns, const fdlbm_transport* tr,
                     const fdlbm_kinetics* kin, const fdlbm_fields* init, const fdlbm_options* opts,
                     fdlbm_handle** out) {
  const int nx = geom->nx, ny = geom->ny, nz = geom->nz;
  if (nz < 4) return fail(FDLBM_EINVAL, "D3Q19: nz must be at least 4 (got %d)", nz);
  if ((long long)nx * ny * nz > (1LL << 29)) return fail(FDLBM_EINVAL, "lattice too large (at most 2^29 nodes)");
  const int* fb = geom->face_bc;
  for (int f = 4; f < 6; ++f)
    if (fb[f] < 0 || fb[f] > 4) return fail(FDLBM_EINVAL, "face_bc[%d] invalid", f);
  if ((fb[4] == FDLBM_FACE_PERIODIC) != (fb[5] == FDLBM_FACE_PERIODIC))
    return fail(FDLBM_EINVAL, "periodic faces must come in pairs");
  if (fb[4] == FDLBM_FACE_INLET || fb[4] == FDLBM_FACE_OUTLET || fb[5] == FDLBM_FACE_INLET ||
      fb[5] == FDLBM_FACE_OUTLET)
    return fail(FDLBM_EINVAL, "inlet only on x-, outlet only on x+");
  if (tr->alpha_s > 1.0 / 6.0) return fail(FDLBM_EINVAL, "alpha_s must be <= 1/6 (explicit FD stability in 3D)");
  if (tr->inlet_profile != FDLBM_PROFILE_PLUG) return fail(FDLBM_EINVAL, "D3Q19: plug inlet only");
  if (geom->wall_u) return fail(FDLBM_EINVAL, "D3Q19: moving walls are not implemented");
  const int storage = opts ? opts->storage : FDLBM_STORAGE_FP32;

  fdlbm_handle* h = new fdlbm_handle();
  h->device = opts ? opts->device : 0;
  DeviceGuard guard(h->device);
  h->stream = opts ? (cudaStream_t)opts->stream : nullptr;
  if (opts) {
    h->ualloc = opts->alloc;
    h->ufree = opts->free;
    h->uctx = opts->alloc_ctx;
  }
  const long n = (long)nx * ny * nz;
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->ns = ns;
  h->dim = 3;
  auto bail = [&](fdlbm_status st) {
    release(h);
    delete h;
    return st;
  };

  // Node classes (gas, inlet, outlet; solid nodes with a gas neighbour along any of the
  // 18 links are interface wall nodes).
  Geo3 G;
  G.nx = nx;
  G.ny = ny;
  G.nz = nz;
  G.px = fb[0] == FDLBM_FACE_PERIODIC;
  G.py = fb[2] == FDLBM_FACE_PERIODIC;
  G.pz = fb[4] == FDLBM_FACE_PERIODIC;
  G.cls.assign(n, GAS);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long k = x + (long)nx * (y + (long)ny * z);
        const uint8_t m = geom->mask[k];
        if (m > 2) return bail(fail(FDLBM_EINVAL, "mask value %d at (%d,%d,%d)", m, x, y, z));
        if (m == FDLBM_MASK_GAS) {
          if (x == 0 && fb[0] == FDLBM_FACE_INLET) G.cls[k] = INLET;
          else if (x == nx - 1 && fb[1] == FDLBM_FACE_OUTLET) G.cls[k] = OUTLET;
          else G.cls[k] = GAS;
        } else {
          G.cls[k] = SOLID;
        }
      }
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long k = x + (long)nx * (y + (long)ny * z);
        if (G.cls[k] != SOLID) continue;
        for (int i = 1; i < Q19; ++i)
          if (G.cls_at(x + H3X[i], y + H3Y[i], z + H3Z[i]) == GAS) G.cls[k] = WALL;
      }
  // Code words; geometry checks.
  std::vector<uint64_t> code(n, 0);
  std::vector<int32_t> walls, solids;
  std::vector<int> gas_z(nz + 1, 0), wall_z(nz + 1, 0);
  long gcount = 0;
  for (int z = 0; z < nz; ++z) {
    gas_z[z] = (int)gcount;
    wall_z[z] = (int)walls.size();
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long k = x + (long)nx * (y + (long)ny * z);
        const uint32_t c = G.cls[k];
        uint64_t w = c;
        if (geom->mask[k] == FDLBM_MASK_CATALYTIC) w |= CATALYTIC_BIT;
        if (c == GAS) {
          ++gcount;
          for (int i = 1; i < Q19; ++i) {
            if (G.at(x + H3X[i], y + H3Y[i], z + H3Z[i]) < 0)
              return bail(fail(FDLBM_EGEOM, "gas node (%d,%d,%d) touches a closed lattice face", x, y, z));
            const uint32_t st = G.stencil(x, y, z, i);
            w |= uint64_t(st) << (STENCIL_SHIFT3 + 3 * (i - 1));
            h->stencil_counts[st]++;
          }
          for (int d = 1; d <= 6; ++d)
            if (G.cls_at(x + H3X[d], y + H3Y[d], z + H3Z[d]) == GAS) w |= 1ull << (NBR_SHIFT3 + d - 1);
        } else if (c == WALL || c == SOLID) {
          if (c == WALL) {
            for (int i = 1; i < Q19; ++i) {
              uint32_t st = ST_NOT_ARRIVAL;
              if (G.cls_at(x - H3X[i], y - H3Y[i], z - H3Z[i]) == GAS) {
                st = G.stencil(x, y, z, i);
                h->stencil_counts[st]++;
              }
              w |= uint64_t(st) << (STENCIL_SHIFT3 + 3 * (i - 1));
            }
            walls.push_back((int32_t)k);
          } else {
            solids.push_back((int32_t)k);
          }
          for (int d = 1; d <= 6; ++d) {
            const uint32_t cn = G.cls_at(x + H3X[d], y + H3Y[d], z + H3Z[d]);
            if (cn == WALL || cn == SOLID) w |= 1ull << (NBR_SHIFT3 + d - 1);
          }
        } else if (c == OUTLET && G.cls[k - 1] != GAS) {
          return bail(fail(FDLBM_EGEOM, "outlet node (%d,%d,%d) has no upstream gas node", x, y, z));
        }
        code[k] = w;
        h->counts[c]++;
      }
  }
  gas_z[nz] = (int)gcount;
  wall_z[nz] = (int)walls.size();
  if (opts && opts->strict_geometry)
    for (long k = 0; k < (long)n; ++k) {
      const uint64_t w = code[k];
      const uint32_t c = node_class3(w);
      if (c != GAS && c != WALL) continue;
      for (int i = 1; i < Q19; ++i) {
        const uint32_t st = stencil_of3(w, i);
        if (st == ST_NONE || st == ST_LIN_S0 || st == ST_LIN_S2)
          return bail(fail(FDLBM_EGEOM, "strict geometry: %s node (%ld,%ld,%ld) pulls direction %d without a "
                           "quadratic stencil (concave corner or narrow gap)", c == GAS ? "gas" : "wall",
                           k % nx, (k / nx) % ny, k / ((long)nx * ny), i));
      }
    }
  std::vector<int32_t> solid_list(walls);
  solid_list.insert(solid_list.end(), solids.begin(), solids.end());

  DevParams& P = h->P;
  P.dim = 3;
  P.nx = nx;
  P.ny = ny;
  P.nz = nz;
  P.n = (int)n;
  P.xoff = XOFF3;
  P.yoff = GHOST3;
  P.zoff = GHOST3;
  P.pitch = (nx + 2 * XOFF3 + 31) / 32 * 32;
  P.slab = (long long)P.pitch * (ny + 2 * GHOST3);
  P.plane = (P.slab * (nz + 2 * GHOST3) + 63) / 64 * 64;
  if ((long long)ns * Q19 * P.plane >= (1LL << 31))
    return bail(fail(FDLBM_EINVAL, "lattice too large: %d species x 19 x %lld padded cells exceed 2^31 elements", ns,
                     (long long)P.plane));
  // Padded code words: ghost cells within GHOST3 of a periodic face carry the wrapped
  // node's word, everything else outside the lattice is OUTSIDE.
  std::vector<uint64_t> pcode((size_t)P.plane, uint64_t(OUTSIDE));
  for (int pz = 0; pz < nz + 2 * GHOST3; ++pz)
    for (int py = 0; py < ny + 2 * GHOST3; ++py)
      for (int px = 0; px < P.pitch; ++px) {
        int x = px - XOFF3, y = py - GHOST3, z = pz - GHOST3;
        if (x < 0 || x >= nx) {
          if (!G.px || x < -GHOST3 || x >= nx + GHOST3) continue;
          x = x < 0 ? x + nx : x - nx;
        }
        if (y < 0 || y >= ny) {
          if (!G.py) continue;
          y = y < 0 ? y + ny : y - ny;
        }
        if (z < 0 || z >= nz) {
          if (!G.pz) continue;
          z = z < 0 ? z + nz : z - nz;
        }
        pcode[(size_t)px + (size_t)py * P.pitch + (size_t)pz * P.slab] = code[x + (long)nx * (y + (long)ny * z)];
      }
  // Gas list in z, y, x order.
  std::vector<int2> gas_list;
  gas_list.reserve((size_t)gcount);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const long k = x + (long)nx * (y + (long)ny * z);
        if (G.cls[k] != GAS) continue;
        const bool near = (G.px && (x < GHOST3 || x >= nx - GHOST3)) || (G.py && (y < GHOST3 || y >= ny - GHOST3)) ||
                          (G.pz && (z < GHOST3 || z >= nz - GHOST3));
        const bool outlet = x + 1 == nx - 1 && G.cls[k + 1] == OUTLET;
        const int aux = int(k) | (outlet ? GAS_AUX_OUTLET : 0) | (near ? GAS_AUX_GHOST : 0);
        const long pk = (x + XOFF3) + (long)(y + GHOST3) * P.pitch + (long)(z + GHOST3) * P.slab;
        gas_list.push_back(make_int2((int)pk, aux));
      }
  P.n_gas = (int)gas_list.size();
  // Step-kernel blocks: per z layer the gas blocks, then the wall blocks of that layer;
  // interior solid blocks last.
  std::vector<int4> blocks;
  auto chunks = [&](int role, int first, int last) {
    for (int s0 = first; s0 < last; s0 += STEP_BLOCK3)
      blocks.push_back(make_int4(role, s0, std::min(STEP_BLOCK3, last - s0), 0));
  };
  for (int z = 0; z < nz; ++z) {
    chunks(0, gas_z[z], gas_z[z + 1]);
    chunks(1, wall_z[z], wall_z[z + 1]);
  }
  chunks(1, (int)walls.size(), (int)solid_list.size());
  P.n_blocks = (int)blocks.size();
  h->blocks_host = blocks;
  P.ns = ns;
  P.periodic_x = G.px;
  P.periodic_y = G.py;
  P.periodic_z = G.pz;
  P.n_solid_list = (int)solid_list.size();
  P.n_wall_list = (int)walls.size();
  for (int f = 0; f < 6; ++f) P.fixedT_face[f] = fb[f] == FDLBM_FACE_FIXED_T;
  set_physics_params(h, species, ns, tr, kin, storage, 3);
  P.ledger_detail = (opts && opts->ledger_detail) ? 1 : 0;
  for (int i = 0; i < Q19; ++i) P.W0_19[i] = (float)wrest3_h(i, h->T_st);

  // Device state.
  fdlbm_status st;
  DevState& S = h->S;
  const size_t pop_bytes = pop_bytes_per_value(storage) * (size_t)ns * Q19 * (size_t)P.plane;
  void* p;
  for (int b = 0; b < 2; ++b) {
    if ((st = dalloc(h, pop_bytes, &p)) != FDLBM_OK) return bail(st);
    S.h[b] = p;
    if ((st = dalloc(h, sizeof(float) * n, &p)) != FDLBM_OK) return bail(st);
    S.Ts[b] = (float*)p;
  }
#define ALLOC3(field, type, count)                                               \
  if ((st = dalloc(h, sizeof(type) * (size_t)(count), &p)) != FDLBM_OK) return bail(st); \
  field = (type*)p;
  ALLOC3(S.code64, uint64_t, P.plane);
  ALLOC3(S.solid_list, int32_t, std::max<size_t>(solid_list.size(), 1));
  ALLOC3(S.gas_list, int2, std::max<size_t>(gas_list.size(), 1));
  ALLOC3(S.blocks, int4, std::max<size_t>(blocks.size(), 1));
  ALLOC3(S.F[0], float, (size_t)(ns + 1) * P.plane);
  ALLOC3(S.F[1], float, (size_t)(ns + 1) * P.plane);
  ALLOC3(S.mom, float, (size_t)(ns + 4) * n);
  ALLOC3(S.Tgas, float, 2 * (size_t)n);
  ALLOC3(S.snap, float, (size_t)(ns + 5) * n);
  ALLOC3(S.ledger, double, (size_t)LG_COUNT * ledger_slots(P));
  ALLOC3(S.rw, float, (size_t)ns * std::max<size_t>(walls.size(), 1));
  ALLOC3(S.flags, int, 4);
  ALLOC3(S.red, double, totals_count(ns) + residual_count3(ns) + LG_COUNT + 8);
  ALLOC3(h->out_buf, float, (size_t)(2 * ns + 5) * n);
#undef ALLOC3
  cudaError_t e = cudaMemcpyAsync(S.code64, pcode.data(), sizeof(uint64_t) * pcode.size(), cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess && !solid_list.empty())
    e = cudaMemcpyAsync(S.solid_list, solid_list.data(), sizeof(int32_t) * solid_list.size(), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess && !blocks.empty())
    e = cudaMemcpyAsync(S.blocks, blocks.data(), sizeof(int4) * blocks.size(), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && !gas_list.empty())
    e = cudaMemcpyAsync(S.gas_list, gas_list.data(), sizeof(int2) * gas_list.size(), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bail(cuda_fail(e, "upload geometry"));
  if ((st = upload_and_init3(h, init)) != FDLBM_OK) return bail(st);
  *out = h;
  return FDLBM_OK;
}

// Initial state of a D3Q19 handle from FP64 host fields (as upload_and_init).
fdlbm_status upload_and_init3(fdlbm_handle* h, const fdlbm_fields* f) {
  const long n = (long)h->nx * h->ny * h->nz;
  const int ns = h->ns;
  const double tl = 1.0 / (3.0 * h->T0);
  std::vector<double> X((size_t)ns * n), u(3 * (size_t)n, 0.0), T(n), Ts(n), C(n, 1.0);
  for (int j = 0; j < ns; ++j)
    for (long k = 0; k < n; ++k) X[(size_t)j * n + k] = (f && f->X) ? f->X[(size_t)j * n + k] : h->X_init[j];
  if (f && f->u) std::memcpy(u.data(), f->u, sizeof(double) * 3 * n);
  for (long k = 0; k < n; ++k) {
    T[k] = (f && f->T_K) ? f->T_K[k] * tl : h->T_init_lat;
    Ts[k] = (f && f->Ts_K) ? f->Ts_K[k] * tl : h->Ts_init_lat;
    if (f && f->C) C[k] = f->C[k];
    if (!(T[k] > 0) || !(C[k] > 0)) return fail(FDLBM_EINVAL, "initial T and C must be positive (node %ld)", k);
  }
  if (fdlbm_status st = check_initial_state(h, X, u, T, n, 3); st != FDLBM_OK) return st;
  // inlet: X_inlet[ns], T_inlet (lattice), u_inlet (plug)
  std::vector<double> inlet(h->X_inlet);
  inlet.push_back(h->T_inlet_lat);
  inlet.push_back(double(h->P.u_inlet));
  const size_t total = X.size() + u.size() + T.size() + Ts.size() + C.size() + inlet.size();
  double* d = nullptr;
  CK(cudaMalloc(&d, sizeof(double) * total), "init staging alloc");
  size_t off = 0;
  double* dX = d + off; off += X.size();
  double* du = d + off; off += u.size();
  double* dT = d + off; off += T.size();
  double* dTs = d + off; off += Ts.size();
  double* dC = d + off; off += C.size();
  double* dIn = d + off;
  cudaError_t e = cudaSuccess;
  auto up = [&](double* dst, const std::vector<double>& v) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, h->stream);
  };
  up(dX, X);
  up(du, u);
  up(dT, T);
  up(dTs, Ts);
  up(dC, C);
  up(dIn, inlet);
  if (e == cudaSuccess) e = launch_init3(h->P, h->S, dX, du, dT, dTs, dC, dIn, h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->S.ledger, 0, sizeof(double) * LG_COUNT * ledger_slots(h->P), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->S.flags, 0, sizeof(int) * 4, h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->S.rw, 0xFF, sizeof(float) * (size_t)ns * std::max(h->P.n_wall_list, 1), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "initialise state");
  h->cur = 0;
  h->steps = 0;
  h->steps_at_residual = 0;
  h->have_snap = false;
  h->mom_fresh = true;
  std::vector<double> tot(totals_count(ns));
  fdlbm_status st = read_totals(h, tot.data());
  if (st != FDLBM_OK) return st;
  h->E0 = tot[0];
  h->H0 = tot[1];
  for (int j = 0; j < ns; ++j) {
    h->mass0[j] = tot[2 + j];
    h->moles0[j] = tot[2 + ns + j];
  }
  h->E_pop0 = 0.0;
  if (h->P.ledger_detail) {
    st = read_pop_energy(h, &h->E_pop0);
    if (st != FDLBM_OK) return st;
  }
  return FDLBM_OK;
}


}  // namespace

extern "C" {

fdlbm_status fdlbm_set_fields(fdlbm_handle* h, const fdlbm_fields* f) {
  if (!h) return fail(FDLBM_EINVAL, "bad handle");
  DeviceGuard guard(h->device);
  return upload_and_init(h, f);
}

fdlbm_status fdlbm_moments(fdlbm_handle* h, float* dst, int dst_on_device) {
  return fdlbm_moments_ex(h, 0u, dst, dst_on_device);
}

fdlbm_status fdlbm_moments_ex(fdlbm_handle* h, unsigned flags, float* dst, int dst_on_device) {
  if (!h || !dst) return fail(FDLBM_EINVAL, "bad handle or destination");
  if (flags & ~unsigned(FDLBM_MOMENTS_T_DEVIATION)) return fail(FDLBM_EINVAL, "unknown moments flags 0x%x", flags);
  const bool t_dev = (flags & FDLBM_MOMENTS_T_DEVIATION) != 0;
  DeviceGuard guard(h->device);
  fdlbm_status st = ensure_moments(h);
  if (st != FDLBM_OK) return st;
  const size_t count = (size_t)(2 * h->ns + 2 + h->dim) * h->nx * h->ny * h->nz;
  auto out = [&](float* d) {
    return h->dim == 3 ? launch_moments_out3(h->P, h->S, h->cur, d, t_dev, h->stream)
                       : launch_moments_out(h->P, h->S, h->cur, d, t_dev, h->stream);
  };
  if (dst_on_device) {
    CK(out(dst), "moments output");
    return FDLBM_OK;
  }
  CK(out(h->out_buf), "moments output");
  CK(cudaMemcpyAsync(dst, h->out_buf, sizeof(float) * count, cudaMemcpyDeviceToHost, h->stream), "copy moments");
  CK(cudaStreamSynchronize(h->stream), "stream sync");
  return FDLBM_OK;
}

fdlbm_status fdlbm_populations(fdlbm_handle* h, float* dst, int dst_on_device) {
  if (!h || !dst) return fail(FDLBM_EINVAL, "bad handle or destination");
  DeviceGuard guard(h->device);
  const size_t count = (size_t)h->ns * (h->dim == 3 ? Q19 : Q) * h->nx * h->ny * h->nz;
  auto out = [&](float* d) {
    return h->dim == 3 ? launch_populations_out3(h->P, h->S, h->cur, d, h->stream)
                       : launch_populations_out(h->P, h->S, h->cur, d, h->stream);
  };
  if (dst_on_device) {
    CK(out(dst), "populations output");
    return FDLBM_OK;
  }
  float* tmp = nullptr;
  CK(cudaMalloc(&tmp, sizeof(float) * count), "staging alloc");
  cudaError_t e = out(tmp);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tmp, sizeof(float) * count, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "populations output");
  return FDLBM_OK;
}

fdlbm_status fdlbm_enthalpy_balance(fdlbm_handle* h, fdlbm_balance* out) {
  if (!h || !out) return fail(FDLBM_EINVAL, "bad handle or output");
  DeviceGuard guard(h->device);
  const int ns = h->ns;
  std::vector<double> tot(totals_count(ns));
  fdlbm_status st = read_totals(h, tot.data());
  if (st != FDLBM_OK) return st;
  double lg[LG_COUNT];
  double* lsum = h->S.red + totals_count(ns) + residual_count3(ns);
  CK(launch_ledger_sum(h->P, h->S, lsum, h->stream), "ledger sum");
  CK(cudaMemcpyAsync(lg, lsum, sizeof(lg), cudaMemcpyDeviceToHost, h->stream), "read ledger");
  CK(cudaStreamSynchronize(h->stream), "stream sync");
  std::memset(out, 0, sizeof(*out));
  out->steps = h->steps;
  out->E_gas = tot[0];
  out->E_gas0 = h->E0;
  out->H_solid = tot[1];
  out->H_solid0 = h->H0;
  out->Q_reaction = lg[LG_QRXN];
  out->Q_wall = lg[LG_QWALL];
  out->Q_couple = lg[LG_QCOUPLE];
  out->Q_fixedT = lg[LG_QFIXEDT];
  out->noconv = lg[LG_NOCONV];
  out->residual = (tot[0] - h->E0) + (tot[1] - h->H0) - lg[LG_QRXN] - lg[LG_QFIXEDT];
  out->solid_residual = (tot[1] - h->H0) - (lg[LG_QRXN] + lg[LG_QCOUPLE] + lg[LG_QFIXEDT]);
  for (int j = 0; j < ns; ++j) {
    out->mass[j] = tot[2 + j];
    out->mass0[j] = h->mass0[j];
    out->moles[j] = tot[2 + ns + j];
    out->moles0[j] = h->moles0[j];
  }
  out->eps_paper = 0.0;
  if (h->eps_species >= 0) {
    const int jr = h->eps_species;
    const double Qco = h->heat0 * (tot[2 + ns + jr] - h->moles0[jr]) / h->eps_nu;
    if (Qco != 0.0) out->eps_paper = ((tot[0] - h->E0) + (tot[1] - h->H0) - Qco) / Qco;
  }
  out->closure = std::nan("");
  if (h->P.ledger_detail) {
    double Ep = 0.0;
    st = read_pop_energy(h, &Ep);
    if (st != FDLBM_OK) return st;
    out->ledger_detail = 1;
    out->E_pop = Ep;
    out->E_pop0 = h->E_pop0;
    out->Q_inlet = lg[LG_QIN];
    out->Q_outlet = lg[LG_QOUT];
    out->D_interp = lg[LG_DINT];
    out->D_collision = lg[LG_DCOL];
    out->D_coupling = lg[LG_QWALLX] + lg[LG_QCOUPLE];
    out->D_solid = lg[LG_DH] - (lg[LG_QRXN] + lg[LG_QCOUPLE] + lg[LG_QFIXEDT]);
    out->closure = (Ep - h->E_pop0) + (tot[1] - h->H0) - lg[LG_QRXN] - lg[LG_QFIXEDT] - out->Q_inlet -
                   out->Q_outlet - out->D_interp - out->D_collision - out->D_coupling - out->D_solid;
  }
  return FDLBM_OK;
}

fdlbm_status fdlbm_residual(fdlbm_handle* h, double* out) {
  if (!h || !out) return fail(FDLBM_EINVAL, "bad handle or output");
  DeviceGuard guard(h->device);
  fdlbm_status st = ensure_moments(h);
  if (st != FDLBM_OK) return st;
  const int ns = h->ns, nf = ns + 2 + h->dim;
  if (h->dim == 3) CK(launch_residual3(h->P, h->S, h->cur, h->stream), "residual launch");
  else CK(launch_residual(h->P, h->S, h->cur, h->stream), "residual launch");
  std::vector<double> sums(h->dim == 3 ? residual_count3(ns) : residual_count(ns));
  CK(cudaMemcpyAsync(sums.data(), h->S.red + totals_count(ns), sizeof(double) * sums.size(),
                     cudaMemcpyDeviceToHost, h->stream),
     "read residual");
  CK(cudaStreamSynchronize(h->stream), "stream sync");
  double r = std::numeric_limits<double>::infinity();
  if (h->have_snap) {
    const double K = double(std::max<int64_t>(h->steps - h->steps_at_residual, 1));
    r = 0.0;
    for (int f = 0; f < nf; ++f) {
      const double dn = std::sqrt(sums[2 * f]), fn = std::sqrt(sums[2 * f + 1]);
      r = std::max(r, dn / (K * std::max(fn, 1e-30)));
    }
  }
  h->have_snap = true;
  h->steps_at_residual = h->steps;
  *out = r;
  return FDLBM_OK;
}

// Address of the static totals scratch, looked up once per device (with that device
// current) and kept for the life of the process. g_static_mu is held from the lookup
// until the call's read-back has completed: calls from several host threads, handles or
// streams then take the scratch one after another instead of racing on it.
namespace {
constexpr int STATIC_MAX_DEVICES = 64;
std::mutex g_static_mu;
double* g_static_scratch[STATIC_MAX_DEVICES] = {};
}  // namespace

fdlbm_status fdlbm_totals_static(fdlbm_handle* h, double* out, int out_len) {
  if (!h || !out) return fail(FDLBM_EINVAL, "bad handle or output");
  if (h->dim != 2) return fail(FDLBM_EINVAL, "the allocation-free totals are implemented for D2Q9 handles only");
  const int ns = h->ns, cnt = totals_count(ns);
  if (out_len < cnt) return fail(FDLBM_EINVAL, "out_len %d < %d (2 + 2 n_species)", out_len, cnt);
  const long long need = totals_static_doubles((long long)h->nx * h->ny, ns) * (long long)sizeof(double);
  if (need > FDLBM_STATIC_SCRATCH_BYTES)
    return fail(FDLBM_EINVAL,
                "lattice %dx%d with %d species needs %lld bytes of static totals scratch, limit %d "
                "(FDLBM_STATIC_SCRATCH_BYTES); use fdlbm_enthalpy_balance",
                h->nx, h->ny, ns, need, FDLBM_STATIC_SCRATCH_BYTES);
  if (h->device < 0 || h->device >= STATIC_MAX_DEVICES)
    return fail(FDLBM_EINVAL, "device %d outside the %d devices the static scratch serves", h->device,
                STATIC_MAX_DEVICES);
  DeviceGuard guard(h->device);
  std::lock_guard<std::mutex> lock(g_static_mu);  // until the stream sync below
  if (!g_static_scratch[h->device]) {
    double* p = nullptr;
    CK(totals_static_scratch(&p), "static totals scratch address");
    g_static_scratch[h->device] = p;
  }
  double* const scratch = g_static_scratch[h->device];
  fdlbm_status st = ensure_moments(h);
  if (st != FDLBM_OK) return st;
  CK(launch_totals_static(h->P, h->S, h->cur, scratch, h->stream), "static totals launch");
  const long long rows = (totals_static_doubles((long long)h->nx * h->ny, ns) / cnt) - 1;
  CK(cudaMemcpyAsync(out, scratch + rows * cnt, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->stream),
     "read static totals");
  CK(cudaStreamSynchronize(h->stream), "stream sync");
  return FDLBM_OK;
}

// Checkpoint file: a fixed header, then the state the next step reads. Layout (native
// little-endian): char magic[8] "FDLBMCK2"; u64 fingerprint; i32 nx, ny, ns, n_blocks;
// i64 plane, steps, steps_at_residual; i32 have_snap, flags; f64 E0, H0, mass0[MAX_NS],
// moles0[MAX_NS], E_pop0; then h[cur] [ns][9][plane] in the storage type, FP32 F[cur] [1 + ns][plane], Ts[cur] [n],
// Tgas[cur] [n], mom [ns + 3][n], snap [ns + 4][n], FP64 ledger [n_blocks][LG_COUNT],
// FP32 wall densities [ns][n_wall_list].
namespace {

constexpr char CK_MAGIC[8] = {'F', 'D', 'L', 'B', 'M', 'C', 'K', '2'};

// FNV-1a over the node code words and the device parameters: a checkpoint loads only
// into a handle built from the same geometry, species, transport and kinetics.
uint64_t fingerprint(const fdlbm_handle* h) {
  uint64_t f = 1469598103934665603ull;
  auto mix = [&f](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) f = (f ^ b[i]) * 1099511628211ull;
  };
  mix(h->code.data(), sizeof(uint32_t) * h->code.size());
  mix(&h->P, sizeof(DevParams));
  return f;
}

struct CkHeader {
  char magic[8];
  uint64_t fp;
  int32_t nx, ny, ns, n_blocks;
  int64_t plane, steps, steps_at_residual;
  int32_t have_snap, flags;
  double E0, H0, mass0[MAX_NS], moles0[MAX_NS], E_pop0;
};

// The device buffers of a checkpoint, in file order: {device pointer, bytes}.
std::vector<std::pair<void*, size_t>> ck_buffers(fdlbm_handle* h) {
  const DevParams& P = h->P;
  const size_t n = (size_t)P.n, ns = (size_t)P.ns, plane = (size_t)P.plane;
  return {{h->S.h[h->cur], pop_bytes_per_value(P.storage) * ns * Q * plane},
          {h->S.Ts[h->cur], sizeof(float) * n},
          {h->S.Tgas + (size_t)h->cur * n, sizeof(float) * n},
          {h->S.mom, sizeof(float) * (ns + 3) * n},
          {h->S.snap, sizeof(float) * (ns + 4) * n},
          {h->S.ledger, sizeof(double) * LG_COUNT * (size_t)ledger_slots(P)},
          {h->S.rw, sizeof(float) * ns * (size_t)std::max(P.n_wall_list, 1)}};
}

}  // namespace

fdlbm_status fdlbm_save(fdlbm_handle* h, const char* path) {
  if (!h || !path) return fail(FDLBM_EINVAL, "bad handle or path");
  if (h->dim != 2) return fail(FDLBM_EINVAL, "checkpoints are implemented for D2Q9 handles only");
  DeviceGuard guard(h->device);
  fdlbm_status st = ensure_moments(h);
  if (st != FDLBM_OK) return st;
  CkHeader hd{};
  std::memcpy(hd.magic, CK_MAGIC, 8);
  hd.fp = fingerprint(h);
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.ns = h->ns;
  hd.n_blocks = ledger_slots(h->P);
  hd.plane = h->P.plane;
  hd.steps = h->steps;
  hd.steps_at_residual = h->steps_at_residual;
  hd.have_snap = h->have_snap ? 1 : 0;
  CK(cudaMemcpyAsync(&hd.flags, h->S.flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read flags");
  hd.E0 = h->E0;
  hd.H0 = h->H0;
  hd.E_pop0 = h->E_pop0;
  std::memcpy(hd.mass0, h->mass0, sizeof(hd.mass0));
  std::memcpy(hd.moles0, h->moles0, sizeof(hd.moles0));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(FDLBM_EIO, "cannot open %s for writing", path);
  bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
  std::vector<unsigned char> buf;
  for (const auto& b : ck_buffers(h)) {
    if (!ok) break;
    buf.resize(b.second);
    const cudaError_t e = cudaMemcpyAsync(buf.data(), b.first, b.second, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && cudaStreamSynchronize(h->stream) == cudaSuccess) {
      ok = std::fwrite(buf.data(), 1, b.second, f) == b.second;
    } else {
      std::fclose(f);
      return cuda_fail(e != cudaSuccess ? e : cudaGetLastError(), "read state for checkpoint");
    }
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(FDLBM_EIO, "short write to %s", path);
  return FDLBM_OK;
}

fdlbm_status fdlbm_load(fdlbm_handle* h, const char* path) {
  if (!h || !path) return fail(FDLBM_EINVAL, "bad handle or path");
  if (h->dim != 2) return fail(FDLBM_EINVAL, "checkpoints are implemented for D2Q9 handles only");
  DeviceGuard guard(h->device);
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(FDLBM_EIO, "cannot open %s", path);
  CkHeader hd{};
  if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, CK_MAGIC, 8) != 0) {
    std::fclose(f);
    return fail(FDLBM_EIO, "%s is not a solver checkpoint", path);
  }
  if (hd.fp != fingerprint(h) || hd.nx != h->nx || hd.ny != h->ny || hd.ns != h->ns ||
      hd.n_blocks != ledger_slots(h->P) || hd.plane != h->P.plane) {
    std::fclose(f);
    return fail(FDLBM_EINVAL,
                "checkpoint %s was written by a solver with another geometry or parameters "
                "(%dx%d, %d species)", path, hd.nx, hd.ny, hd.ns);
  }
  CK(cudaStreamSynchronize(h->stream), "stream sync");
  std::vector<unsigned char> buf;
  for (const auto& b : ck_buffers(h)) {
    buf.resize(b.second);
    if (std::fread(buf.data(), 1, b.second, f) != b.second) {
      std::fclose(f);
      return fail(FDLBM_EIO, "%s is truncated", path);
    }
    const cudaError_t e = cudaMemcpyAsync(b.first, buf.data(), b.second, cudaMemcpyHostToDevice, h->stream);
    const cudaError_t e2 = e == cudaSuccess ? cudaStreamSynchronize(h->stream) : e;
    if (e2 != cudaSuccess) {
      std::fclose(f);
      return cuda_fail(e2, "write checkpoint state");
    }
  }
  std::fclose(f);
  // The other population copy: nodes the step never rewrites (inlet) keep their values.
  const size_t pop_bytes = pop_bytes_per_value(h->P.storage) * (size_t)h->ns * Q * (size_t)h->P.plane;
  CK(cudaMemcpyAsync(h->S.h[h->cur ^ 1], h->S.h[h->cur], pop_bytes, cudaMemcpyDeviceToDevice, h->stream),
     "copy populations");
  CK(cudaMemcpyAsync(h->S.flags, &hd.flags, sizeof(int), cudaMemcpyHostToDevice, h->stream), "write flags");
  CK(cudaStreamSynchronize(h->stream), "stream sync");
  h->steps = hd.steps;
  h->steps_at_residual = hd.steps_at_residual;
  h->have_snap = hd.have_snap != 0;
  h->mom_fresh = true;
  h->E0 = hd.E0;
  h->H0 = hd.H0;
  h->E_pop0 = hd.E_pop0;
  std::memcpy(h->mass0, hd.mass0, sizeof(hd.mass0));
  std::memcpy(h->moles0, hd.moles0, sizeof(hd.moles0));
  return FDLBM_OK;
}

fdlbm_status fdlbm_info(const fdlbm_handle* h, fdlbm_info_t* out) {
  if (!h || !out) return fail(FDLBM_EINVAL, "bad handle or output");
  std::memset(out, 0, sizeof(*out));
  out->n_nodes = (int64_t)h->nx * h->ny * h->nz;
  out->n_gas = h->counts[GAS];
  out->n_inlet = h->counts[INLET];
  out->n_outlet = h->counts[OUTLET];
  out->n_wall = h->counts[WALL];
  out->n_solid = h->counts[SOLID];
  for (int c = 0; c < 6; ++c) out->stencil_counts[c] = h->stencil_counts[c];
  out->ns = h->ns;
  out->T_ref_lat = h->T_inlet_lat;
  out->steps = h->steps;
  out->device_bytes = h->bytes;
  return FDLBM_OK;
}

fdlbm_status fdlbm_profile(fdlbm_handle* h, int enable) {
  if (!h) return fail(FDLBM_EINVAL, "bad handle");
  DeviceGuard guard(h->device);
  if (enable && h->events.empty()) {
    h->events.resize(2 * 65536);
    for (auto& e : h->events) CK(cudaEventCreate(&e), "event create");
  }
  h->profiling = enable != 0;
  h->events_used = 0;
  return FDLBM_OK;
}

fdlbm_status fdlbm_kernel_times(fdlbm_handle* h, double* ms_out2, int64_t* steps_out) {
  if (!h || !ms_out2) return fail(FDLBM_EINVAL, "bad handle or output");
  DeviceGuard guard(h->device);
  CK(cudaStreamSynchronize(h->stream), "stream sync");
  double step = 0.0;
  for (size_t k = 0; k + 2 <= h->events_used; k += 2) {
    float a = 0.f;
    CK(cudaEventElapsedTime(&a, h->events[k], h->events[k + 1]), "event time");
    step += a;
  }
  ms_out2[0] = step;
  ms_out2[1] = 0.0;
  if (steps_out) *steps_out = (int64_t)(h->events_used / 2);
  h->events_used = 0;
  return FDLBM_OK;
}

}  // extern "C"

// A batch steps several handles in one launch per step; see fdlbm.h.
struct fdlbm_batch {
  std::vector<fdlbm_handle*> members;
  int device = 0;
  cudaStream_t stream = nullptr;
  int ns = 0, energy_correction = 0, storage = 0;
  DevParams* d_params = nullptr;
  DevState* d_states = nullptr;
  int2* d_members = nullptr;
  int4* d_blocks = nullptr;
  uint32_t* d_counter = nullptr;
  int n_blocks = 0;
  int64_t counter = 0;                       // steps since d_members was written
  std::vector<int> cur0;                     // member buffers of time level t at counter 0
  std::vector<int64_t> step0;                // member step counts at counter 0
  cudaGraphExec_t graph = nullptr;           // BATCH_GRAPH_STEPS batched steps
  cudaEvent_t done = nullptr;
};

namespace {

constexpr int BATCH_GRAPH_STEPS = 16;

void batch_free_device(fdlbm_batch* b) {
  cudaFree(b->d_params);
  cudaFree(b->d_states);
  cudaFree(b->d_members);
  cudaFree(b->d_blocks);
  cudaFree(b->d_counter);
  b->d_params = nullptr;
  b->d_states = nullptr;
  b->d_members = nullptr;
  b->d_blocks = nullptr;
  b->d_counter = nullptr;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

// (Re)build the device tables of the batch from its members' current state: parameters,
// buffers, the members' time levels and step counts, and the concatenated block tables.
fdlbm_status batch_upload(fdlbm_batch* b) {
  batch_free_device(b);
  const size_t m = b->members.size();
  std::vector<DevParams> params(m);
  std::vector<DevState> states(m);
  std::vector<int2> mem(m);
  std::vector<int4> blocks;
  b->cur0.resize(m);
  b->step0.resize(m);
  for (size_t i = 0; i < m; ++i) {
    fdlbm_handle* h = b->members[i];
    params[i] = h->P;
    states[i] = h->S;
    b->cur0[i] = h->cur;
    b->step0[i] = h->steps;
    mem[i] = make_int2(h->cur, int(uint32_t(h->steps)));
    for (size_t q = 0; q < h->blocks_host.size(); ++q) {
      const int4 d = h->blocks_host[q];
      // gas tiles keep their map row stride; solid blocks take their ledger slot
      blocks.push_back(make_int4(int(2 * i) + d.x, d.y, d.z, d.x == 0 ? d.w : int(q)));
    }
  }
  b->n_blocks = (int)blocks.size();
  b->counter = 0;
  CK(cudaMalloc(&b->d_params, sizeof(DevParams) * std::max<size_t>(m, 1)), "batch allocation");
  CK(cudaMalloc(&b->d_states, sizeof(DevState) * std::max<size_t>(m, 1)), "batch allocation");
  CK(cudaMalloc(&b->d_members, sizeof(int2) * std::max<size_t>(m, 1)), "batch allocation");
  CK(cudaMalloc(&b->d_blocks, sizeof(int4) * std::max<size_t>(blocks.size(), 1)), "batch allocation");
  CK(cudaMalloc(&b->d_counter, sizeof(uint32_t)), "batch allocation");
  if (m) {
    CK(cudaMemcpy(b->d_params, params.data(), sizeof(DevParams) * m, cudaMemcpyHostToDevice), "batch upload");
    CK(cudaMemcpy(b->d_states, states.data(), sizeof(DevState) * m, cudaMemcpyHostToDevice), "batch upload");
    CK(cudaMemcpy(b->d_members, mem.data(), sizeof(int2) * m, cudaMemcpyHostToDevice), "batch upload");
  }
  if (!blocks.empty())
    CK(cudaMemcpy(b->d_blocks, blocks.data(), sizeof(int4) * blocks.size(), cudaMemcpyHostToDevice), "batch upload");
  CK(cudaMemset(b->d_counter, 0, sizeof(uint32_t)), "batch upload");
  return FDLBM_OK;
}

BatchLaunch batch_launch_args(const fdlbm_batch* b) {
  BatchLaunch B;
  B.params = b->d_params;
  B.states = b->d_states;
  B.members = b->d_members;
  B.blocks = b->d_blocks;
  B.counter = b->d_counter;
  B.n_blocks = b->n_blocks;
  B.ns = b->ns;
  B.energy_correction = b->energy_correction;
  B.storage = b->storage;
  return B;
}

// The members' streams wait for `from`'s work so far.
fdlbm_status streams_wait(cudaStream_t from, cudaEvent_t ev, const std::vector<fdlbm_handle*>& to) {
  CK(cudaEventRecord(ev, from), "event record");
  for (fdlbm_handle* h : to) CK(cudaStreamWaitEvent(h->stream, ev, 0), "stream wait");
  return FDLBM_OK;
}

}  // namespace

extern "C" {

fdlbm_status fdlbm_batch_create(fdlbm_handle* const* handles, int n, fdlbm_batch** out) {
  if (!out || !handles || n < 1) return fail(FDLBM_EINVAL, "need an output pointer and at least one handle");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!handles[i]) return fail(FDLBM_EINVAL, "handle %d is NULL", i);
    if (handles[i]->dim != 2) return fail(FDLBM_EINVAL, "batches are implemented for D2Q9 handles only");
    if (handles[i]->P.local_tau) return fail(FDLBM_EINVAL, "batches do not take handles with local relaxation times");
    if (handles[i]->P.ledger_detail) return fail(FDLBM_EINVAL, "batches do not take handles that keep exact accounts");
    for (int q = 0; q < i; ++q)
      if (handles[q] == handles[i]) return fail(FDLBM_EINVAL, "handle %d appears twice", i);
    const fdlbm_handle* h = handles[i];
    const fdlbm_handle* h0 = handles[0];
    if (h->device != h0->device || h->ns != h0->ns || h->P.storage != h0->P.storage ||
        h->P.energy_correction != h0->P.energy_correction)
      return fail(FDLBM_EINVAL,
                  "handle %d differs from handle 0 in device, species count, storage or energy correction", i);
  }
  DeviceGuard guard(handles[0]->device);
  fdlbm_batch* b = new fdlbm_batch;
  b->members.assign(handles, handles + n);
  b->device = handles[0]->device;
  b->ns = handles[0]->ns;
  b->energy_correction = handles[0]->P.energy_correction;
  b->storage = handles[0]->P.storage;
  // Its own stream: graphs cannot be captured on the legacy default stream the members
  // may use; events order it against the members' streams.
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return cuda_fail(e, "batch stream");
  }
  for (fdlbm_handle* h : b->members) {
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      cudaEventDestroy(b->done);
      cudaStreamDestroy(b->stream);
      delete b;
      return cuda_fail(e, "stream sync");
    }
  }
  fdlbm_status st = batch_upload(b);
  if (st != FDLBM_OK) {
    fdlbm_batch_destroy(b);
    return st;
  }
  *out = b;
  return FDLBM_OK;
}

fdlbm_status fdlbm_batch_step(fdlbm_batch* b, int64_t n) {
  if (!b || n < 0) return fail(FDLBM_EINVAL, "bad batch or step count");
  if (n == 0 || b->members.empty()) return FDLBM_OK;
  DeviceGuard guard(b->device);
  // A member stepped on its own since the tables were written: write them again.
  for (size_t i = 0; i < b->members.size(); ++i) {
    const fdlbm_handle* h = b->members[i];
    if (h->steps != b->step0[i] + b->counter || h->cur != (b->cur0[i] ^ int(b->counter & 1))) {
      for (fdlbm_handle* m : b->members) CK(cudaStreamSynchronize(m->stream), "stream sync");
      CK(cudaStreamSynchronize(b->stream), "stream sync");
      fdlbm_status st = batch_upload(b);
      if (st != FDLBM_OK) return st;
      break;
    }
  }
  // The batch's stream waits for work queued on the members' streams.
  for (fdlbm_handle* h : b->members) {
    CK(cudaEventRecord(b->done, h->stream), "event record");
    CK(cudaStreamWaitEvent(b->stream, b->done, 0), "stream wait");
  }
  const BatchLaunch B = batch_launch_args(b);
  int64_t left = n;
  if (left >= BATCH_GRAPH_STEPS) {
    if (!b->graph) {
      // one plain launch first: it sets the kernel's shared-memory attribute outside
      // the capture
      CK(launch_batch_step(B, b->stream), "batch step");
      --left;
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      cudaError_t e = cudaSuccess;
      for (int q = 0; q < BATCH_GRAPH_STEPS && e == cudaSuccess; ++q) e = launch_batch_step(B, b->stream);
      const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e != cudaSuccess ? e : e2, "capture batch steps");
      }
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        return cuda_fail(e, "instantiate batch graph");
      }
    }
    for (; left >= BATCH_GRAPH_STEPS; left -= BATCH_GRAPH_STEPS) CK(cudaGraphLaunch(b->graph, b->stream), "graph launch");
  }
  for (; left > 0; --left) CK(launch_batch_step(B, b->stream), "batch step");
  b->counter += n;
  for (fdlbm_handle* h : b->members) {
    h->steps += n;
    h->cur ^= int(n & 1);
    h->mom_fresh = false;
  }
  return streams_wait(b->stream, b->done, b->members);
}

fdlbm_status fdlbm_batch_remove(fdlbm_batch* b, fdlbm_handle* h) {
  if (!b || !h) return fail(FDLBM_EINVAL, "bad batch or handle");
  auto it = std::find(b->members.begin(), b->members.end(), h);
  if (it == b->members.end()) return fail(FDLBM_EINVAL, "handle is not a member of the batch");
  DeviceGuard guard(b->device);
  CK(cudaStreamSynchronize(b->stream), "stream sync");
  b->members.erase(it);
  return batch_upload(b);
}

int fdlbm_batch_size(const fdlbm_batch* b) { return b ? (int)b->members.size() : 0; }

void fdlbm_batch_destroy(fdlbm_batch* b) {
  if (!b) return;
  {
    DeviceGuard guard(b->device);
    cudaStreamSynchronize(b->stream);
    batch_free_device(b);
    if (b->done) cudaEventDestroy(b->done);
    if (b->stream) cudaStreamDestroy(b->stream);
  }
  delete b;
}

void fdlbm_destroy(fdlbm_handle* h) {
  if (!h) return;
  {
    DeviceGuard guard(h->device);
    cudaStreamSynchronize(h->stream);
    for (auto& e : h->events) cudaEventDestroy(e);
    release(h);
  }
  delete h;
}

}  // extern "C"
