// CUDA kernels of the coupled FD-LBM solver (sm_103a).
//
// Storage: populations are FP32 deviations h = g - rref_j W0_i from the rest equilibrium
// of the inlet state (rref_j = X_inlet,j M_j, W0 = f^eq(1, 0, T_ref)); the solid
// temperature is stored as T_s - T_ref. Every moment and equilibrium is evaluated in
// that deviation form, so FP32 keeps the precision the FP64 reference needs.
//
// Per time step (all kernels read time level t only):
//   solid_kernel: interface (wall) nodes stream in the populations arriving from the gas,
//     iterate the wall density with the surface reaction (Sec. 4.3, Eq. BC_gji), emit
//     the unknown populations and apply the FD heat step with the interface coupling and
//     the reaction heat (Sec. 5); interior solid nodes apply the FD step only.
//   gas_kernel: fused pull streaming with the off-lattice interpolation (Sec. 4.2),
//     moments (Eq. moments_of_g), energy-correction divergence on a shared-memory tile
//     with a recomputed one-node halo, two-step collision (Eq. final_kinetic_equation),
//     outlet equilibrium.
#include <cfloat>
#include <cmath>

#include "fdlbm_internal.h"

namespace fdlbm {

namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int HALO_N = 2 * (TX + 2) + 2 * TY;

__host__ __device__ constexpr int EX(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0; }
__host__ __device__ constexpr int EY(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0; }
__host__ __device__ constexpr int OPP(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5); }
// Forcing coefficients of Eq. psi_jialpha times 4 c_j.
__host__ __device__ constexpr float PSX(int i) { return i == 1 ? 4.f : i == 3 ? -4.f : (i == 5 || i == 8) ? -1.f : (i == 6 || i == 7) ? 1.f : 0.f; }
__host__ __device__ constexpr float PSY(int i) { return i == 2 ? 4.f : i == 4 ? -4.f : (i == 5 || i == 6) ? -1.f : (i == 7 || i == 8) ? 1.f : 0.f; }

// Linear index of (x, y), wrapped on periodic axes; -1 off the lattice.
__device__ __forceinline__ int lat_index(const DevParams& P, int x, int y) {
  if (x < 0) { if (!P.periodic_x) return -1; x += P.nx; }
  else if (x >= P.nx) { if (!P.periodic_x) return -1; x -= P.nx; }
  if (y < 0) { if (!P.periodic_y) return -1; y += P.ny; }
  else if (y >= P.ny) { if (!P.periodic_y) return -1; y -= P.ny; }
  return x + P.nx * y;
}

// Tile cells resolve only positions at most one node off the lattice (a single wrap on
// periodic axes); farther cells of a ragged tile are never read and stay empty.
__device__ __forceinline__ int cell_index(const DevParams& P, int x, int y) {
  if (x < -1 || x > P.nx || y < -1 || y > P.ny) return -1;
  return lat_index(P, x, y);
}

// Interpolation weights of the stencils (Eqs. interpol_bulk, interpol_away,
// interpol_towards expanded into weights of the streamed off-lattice values).
struct Weights { float c2, c1, c0, f1, f0, fp, b1, b2, b3, a; };
__device__ __forceinline__ Weights weights_of(float a) {
  Weights w;
  float aa = a * a;
  w.c2 = 0.5f * (aa - a); w.c1 = 1.f - aa; w.c0 = 0.5f * (aa + a);
  w.f1 = 1.f - 1.5f * a + 0.5f * aa; w.f0 = 2.f * a - aa; w.fp = 0.5f * (aa - a);
  w.b1 = 1.f + 1.5f * a + 0.5f * aa; w.b2 = -2.f * a - aa; w.b3 = 0.5f * (a + aa);
  w.a = a;
  return w;
}

// Pull one non-rest population of species j into target (x, y) along direction i.
template <int I>
__device__ __forceinline__ float pull_dir(const DevParams& P, const float* __restrict__ pl, int x, int y,
                                          int n, uint32_t st, bool onlat, const Weights& w) {
  constexpr int ex = EX(I), ey = EY(I);
  float s1 = __ldg(pl + lat_index(P, x - ex, y - ey));
  if (onlat) return s1;
  switch (st) {
    case ST_CENTRAL: {
      float s2 = __ldg(pl + lat_index(P, x - 2 * ex, y - 2 * ey));
      float s0 = __ldg(pl + n);
      return fmaf(w.c2, s2, fmaf(w.c1, s1, w.c0 * s0));
    }
    case ST_FORWARD: {
      float s0 = __ldg(pl + n);
      float sp = __ldg(pl + lat_index(P, x + ex, y + ey));
      return fmaf(w.f1, s1, fmaf(w.f0, s0, w.fp * sp));
    }
    case ST_BACKWARD: {
      float s2 = __ldg(pl + lat_index(P, x - 2 * ex, y - 2 * ey));
      float s3 = __ldg(pl + lat_index(P, x - 3 * ex, y - 3 * ey));
      return fmaf(w.b1, s1, fmaf(w.b2, s2, w.b3 * s3));
    }
    case ST_LIN_S0: {
      float s0 = __ldg(pl + n);
      return fmaf(w.a, s0 - s1, s1);
    }
    case ST_LIN_S2: {
      float s2 = __ldg(pl + lat_index(P, x - 2 * ex, y - 2 * ey));
      return fmaf(w.a, s1 - s2, s1);
    }
    default:
      return s1;
  }
}

template <int NS, int I>
__device__ __forceinline__ void pull_species_dir(const DevParams& P, const float* __restrict__ src, int x,
                                                 int y, int n, uint32_t cw, float (&hv)[NS][Q]) {
  uint32_t st = stencil_of(cw, I);
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const float* pl = src + (long long)(j * Q + I) * P.plane;
    Weights w = weights_of(P.a[j]);
    hv[j][I] = pull_dir<I>(P, pl, x, y, n, st, P.onlattice[j] != 0, w);
  }
}

// Stream every population of species 0..NS-1 into gas node (x, y) (index n).
template <int NS>
__device__ __forceinline__ void pull_node(const DevParams& P, const float* __restrict__ src, int x, int y,
                                          int n, uint32_t cw, float (&hv)[NS][Q]) {
#pragma unroll
  for (int j = 0; j < NS; ++j) hv[j][0] = __ldg(src + (long long)(j * Q) * P.plane + n);
  pull_species_dir<NS, 1>(P, src, x, y, n, cw, hv);
  pull_species_dir<NS, 2>(P, src, x, y, n, cw, hv);
  pull_species_dir<NS, 3>(P, src, x, y, n, cw, hv);
  pull_species_dir<NS, 4>(P, src, x, y, n, cw, hv);
  pull_species_dir<NS, 5>(P, src, x, y, n, cw, hv);
  pull_species_dir<NS, 6>(P, src, x, y, n, cw, hv);
  pull_species_dir<NS, 7>(P, src, x, y, n, cw, hv);
  pull_species_dir<NS, 8>(P, src, x, y, n, cw, hv);
}

// Runtime-direction pull used on wall nodes (few, divergent anyway).
__device__ float pull_rt(const DevParams& P, const float* __restrict__ src, int j, int i, int x, int y,
                         int n, uint32_t st) {
  const float* pl = src + (long long)(j * Q + i) * P.plane;
  Weights w = weights_of(P.a[j]);
  bool onlat = P.onlattice[j] != 0;
  switch (i) {
    case 1: return pull_dir<1>(P, pl, x, y, n, st, onlat, w);
    case 2: return pull_dir<2>(P, pl, x, y, n, st, onlat, w);
    case 3: return pull_dir<3>(P, pl, x, y, n, st, onlat, w);
    case 4: return pull_dir<4>(P, pl, x, y, n, st, onlat, w);
    case 5: return pull_dir<5>(P, pl, x, y, n, st, onlat, w);
    case 6: return pull_dir<6>(P, pl, x, y, n, st, onlat, w);
    case 7: return pull_dir<7>(P, pl, x, y, n, st, onlat, w);
    default: return pull_dir<8>(P, pl, x, y, n, st, onlat, w);
  }
}

// Moments of the pulled deviations: species densities, momenta and the g-temperature
// deviation dTg = T_g - T_ref (Eq. moments_of_g, Eq. moments_of_f).
template <int NS>
struct Mom {
  float drho[NS], rho[NS], Jx[NS], Jy[NS];
  float r, jx, jy, C, dTg;
};

template <int NS>
__device__ __forceinline__ void moments(const DevParams& P, const float (&hv)[NS][Q], Mom<NS>& m) {
  m.r = 0.f; m.jx = 0.f; m.jy = 0.f; m.C = 0.f;
  float de = 0.f;
  const float t2 = 2.f * P.Tref;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    float dr = 0.f, ax = 0.f, ay = 0.f, e = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float v = hv[j][i];
      dr += v;
      if (EX(i) != 0) ax += EX(i) > 0 ? v : -v;
      if (EY(i) != 0) ay += EY(i) > 0 ? v : -v;
      e = fmaf(float(EX(i) * EX(i) + EY(i) * EY(i)) - t2, v, e);
    }
    m.drho[j] = dr;
    m.rho[j] = P.rref[j] + dr;
    m.Jx[j] = P.c[j] * ax;
    m.Jy[j] = P.c[j] * ay;
    m.r += m.rho[j];
    m.jx += m.Jx[j];
    m.jy += m.Jy[j];
    m.C = fmaf(m.rho[j], P.invM[j], m.C);
    de = fmaf(P.c2[j], e, de);
  }
  m.dTg = (de - (m.jx * m.jx + m.jy * m.jy) / m.r) / (2.f * m.C);
}

// One Cartesian factor of the product-form equilibrium (Eq. eq_state_pop, positive-sign
// form) and its deviation from the rest factor at T_ref.
__device__ __forceinline__ float wfac(int e, float sv, float Mv2, float T) {
  return e == 0 ? 1.f - Mv2 - T : 0.5f * (float(e) * sv + Mv2 + T);
}
__device__ __forceinline__ float dwfac(int e, float sv, float Mv2, float dT) {
  return e == 0 ? -(Mv2 + dT) : 0.5f * (float(e) * sv + Mv2 + dT);
}
__device__ __forceinline__ float w0fac(int e, float Tref) { return e == 0 ? 1.f - Tref : 0.5f * Tref; }

// Deviation of rho W(e; u) from rref W0(e): (rho - rref) W + rref (dWx Wy + W0x dWy).
struct EqFactors {
  float wx[3], wy[3], dwx[3], dwy[3];  // index e + 1
};
__device__ __forceinline__ void eq_factors(float sqrtM, float M, float ux, float uy, float T, float dT,
                                           EqFactors& f) {
  float sx = sqrtM * ux, sy = sqrtM * uy, mx = M * ux * ux, my = M * uy * uy;
#pragma unroll
  for (int e = -1; e <= 1; ++e) {
    f.wx[e + 1] = wfac(e, sx, mx, T);
    f.wy[e + 1] = wfac(e, sy, my, T);
    f.dwx[e + 1] = dwfac(e, sx, mx, dT);
    f.dwy[e + 1] = dwfac(e, sy, my, dT);
  }
}
__device__ __forceinline__ float eq_dev(const EqFactors& f, int i, float drho, float rref, float Tref) {
  int a = EX(i) + 1, b = EY(i) + 1;
  return drho * f.wx[a] * f.wy[b] + rref * (f.dwx[a] * f.wy[b] + w0fac(EX(i), Tref) * f.dwy[b]);
}

template <int NS>
__device__ __forceinline__ void flag_bad(int* flags, const Mom<NS>& m, float T) {
  if (!(m.r > 0.f) || !(T > 0.f) || !isfinite(m.jx + m.jy + T)) atomicOr(flags, 1);
}

// ---------------------------------------------------------------------------------------
// Gas kernel
// ---------------------------------------------------------------------------------------
// MODE 0: full step (collide, write populations). MODE 1: moments only (no population
// writes; writes mom[]).
template <int NS, bool PHI, int MODE>
__global__ void __launch_bounds__(TX * TY) gas_kernel(DevParams P, const float* __restrict__ src,
                                                      float* __restrict__ dst,
                                                      const uint32_t* __restrict__ code, float* __restrict__ mom,
                                                      float* __restrict__ Tgas, int* __restrict__ flags) {
  __shared__ float s_dT[TY + 2][TX + 2];
  __shared__ float s_K[PHI ? NS : 1][TY + 2][TX + 2];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool own = gx < P.nx && gy < P.ny;
  // Interior cells beyond a ragged edge hold the wrapped node on periodic axes so that
  // the owners' neighbour reads find it.
  const int n = own ? gx + P.nx * gy : cell_index(P, gx, gy);
  const uint32_t cw = n >= 0 ? __ldg(code + n) : uint32_t(OUTSIDE);
  const bool gas = n >= 0 && node_class(cw) == GAS;
  const int wx = n >= 0 ? n % P.nx : 0, wy = n >= 0 ? n / P.nx : 0;

  float hv[NS][Q];
  Mom<NS> m;
  if (gas) {
    pull_node<NS>(P, src, wx, wy, n, cw, hv);
    moments<NS>(P, hv, m);
  }
  if (PHI) {
    s_dT[ty + 1][tx + 1] = gas ? m.dTg : 0.f;
#pragma unroll
    for (int j = 0; j < NS; ++j)
      s_K[j][ty + 1][tx + 1] = gas ? P.kcoef[j] * (m.rho[j] * P.invM[j]) * (P.Tref + m.dTg) : 0.f;
    const int t = ty * TX + tx;
    if (t < HALO_N) {
      int hx, hy;
      if (t < TX + 2) { hx = t - 1; hy = -1; }
      else if (t < 2 * (TX + 2)) { hx = t - (TX + 2) - 1; hy = TY; }
      else if (t < 2 * (TX + 2) + TY) { hx = -1; hy = t - 2 * (TX + 2); }
      else { hx = TX; hy = t - 2 * (TX + 2) - TY; }
      const int hn = cell_index(P, x0 + hx, y0 + hy);
      const uint32_t hcw = hn >= 0 ? __ldg(code + hn) : uint32_t(OUTSIDE);
      float hdT = 0.f, hK[NS];
#pragma unroll
      for (int j = 0; j < NS; ++j) hK[j] = 0.f;
      if (hn >= 0 && node_class(hcw) == GAS) {
        float hh[NS][Q];
        Mom<NS> hm;
        pull_node<NS>(P, src, hn % P.nx, hn / P.nx, hn, hcw, hh);
        moments<NS>(P, hh, hm);
        hdT = hm.dTg;
#pragma unroll
        for (int j = 0; j < NS; ++j) hK[j] = P.kcoef[j] * (hm.rho[j] * P.invM[j]) * (P.Tref + hm.dTg);
      }
      s_dT[hy + 1][hx + 1] = hdT;
#pragma unroll
      for (int j = 0; j < NS; ++j) s_K[j][hy + 1][hx + 1] = hK[j];
    }
    __syncthreads();
  }
  if (!own || !gas) return;

  // Divergence of the energy-correction flux K_j grad T on the 4 axis neighbours: faces
  // to non-gas nodes carry no flux (their K is stored as 0 and their face is skipped).
  float divq[NS];
  float sdq = 0.f;
#pragma unroll
  for (int j = 0; j < NS; ++j) divq[j] = 0.f;
  if (PHI) {
    const float Tc = s_dT[ty + 1][tx + 1];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int ox = d == 0 ? 1 : d == 1 ? -1 : 0;
      const int oy = d == 2 ? 1 : d == 3 ? -1 : 0;
      const int nn = lat_index(P, gx + ox, gy + oy);
      const bool ngas = nn >= 0 && node_class(__ldg(code + nn)) == GAS;
      if (!ngas) continue;
      const float Tn = s_dT[ty + 1 + oy][tx + 1 + ox];
#pragma unroll
      for (int j = 0; j < NS; ++j)
        divq[j] += 0.5f * (s_K[j][ty + 1][tx + 1] + s_K[j][ty + 1 + oy][tx + 1 + ox]) * (Tn - Tc);
    }
#pragma unroll
    for (int j = 0; j < NS; ++j) sdq += divq[j];
  }

  const float ux = m.jx / m.r, uy = m.jy / m.r;
  const float dT = m.dTg + sdq / (4.f * m.C);
  const float T = P.Tref + dT;

  if (MODE == 1 || Tgas != nullptr) {
    if (MODE == 1) {
#pragma unroll
      for (int j = 0; j < NS; ++j) mom[(long long)j * P.n + n] = m.rho[j];
      mom[(long long)NS * P.n + n] = ux;
      mom[(long long)(NS + 1) * P.n + n] = uy;
      mom[(long long)(NS + 2) * P.n + n] = T;
    }
    if (Tgas != nullptr) Tgas[n] = T;
  }
  if (MODE == 1) return;
  flag_bad<NS>(flags, m, T);

  // Corrective diffusion velocity (reading R3: weights 1/(tau2 + 1/2)).
  float nx_ = 0.f, ny_ = 0.f, den = 0.f;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    nx_ = fmaf(P.uc_w[j], m.Jx[j] - m.rho[j] * ux, nx_);
    ny_ = fmaf(P.uc_w[j], m.Jy[j] - m.rho[j] * uy, ny_);
    den = fmaf(P.uc_w[j], m.rho[j], den);
  }
  const float Ucx = nx_ / den, Ucy = ny_ / den;

#pragma unroll
  for (int j = 0; j < NS; ++j) {
    // f-momentum of the species (Eq. moments_of_g, second line) and its velocity,
    // limited for trace species (reading R15).
    const float Jfx = (m.Jx[j] + P.a2[j] * m.rho[j] * (ux + Ucx)) * P.inv1a2[j];
    const float Jfy = (m.Jy[j] + P.a2[j] * m.rho[j] * (uy + Ucy)) * P.inv1a2[j];
    float ujx = ux, ujy = uy;
    if (m.rho[j] != 0.f) {
      const float lim = sqrtf(fmaxf(1.f - T, 0.f) * P.invM[j]);
      ujx = fminf(fmaxf(Jfx / m.rho[j], -lim), lim);
      ujy = fminf(fmaxf(Jfy / m.rho[j], -lim), lim);
    }
    EqFactors fe, fs;
    eq_factors(P.sqrtM[j], P.M[j], ux, uy, T, dT, fe);
    eq_factors(P.sqrtM[j], P.M[j], ujx, ujy, T, dT, fs);
    const float om = P.omega[j], omt = P.omega[j] * P.t1t2[j], wt1 = P.wt1[j];
    const float psi_s = m.rho[j] * P.invtau2[j] * 0.25f / P.c[j];
    const float phi_s = P.M[j] * divq[j];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float feq = eq_dev(fe, i, m.drho[j], P.rref[j], P.Tref);
      const float fst = eq_dev(fs, i, m.drho[j], P.rref[j], P.Tref);
      float force = psi_s * (PSX(i) * Ucx + PSY(i) * Ucy);
      if (i == 0) force -= phi_s;
      else if (i <= 4) force += 0.25f * phi_s;
      const float h = hv[j][i];
      const float hn = h - om * (h - fst) - omt * (fst - feq) + wt1 * force;
      dst[(long long)(j * Q + i) * P.plane + n] = hn;
    }
  }

  // Outlet (reading R13): equilibrium at the outlet pressure with this node's
  // composition, velocity and temperature.
  if (gx + 1 < P.nx && !P.periodic_x && node_class(__ldg(code + n + 1)) == OUTLET) {
    const float Cout = P.p_out / T;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      EqFactors fe;
      eq_factors(P.sqrtM[j], P.M[j], ux, uy, T, dT, fe);
      const float rj = m.rho[j] * P.invM[j] / m.C * Cout * P.M[j];
      const float dr = rj - P.rref[j];
#pragma unroll
      for (int i = 0; i < Q; ++i)
        dst[(long long)(j * Q + i) * P.plane + n + 1] = eq_dev(fe, i, dr, P.rref[j], P.Tref);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Wall + solid kernel
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float wrest(int i, float T) {
  return (EX(i) == 0 ? 1.f - T : 0.5f * T) * (EY(i) == 0 ? 1.f - T : 0.5f * T);
}

__device__ void rates(const DevParams& P, const float* rw, float Tw, float* rate) {
  float Cw[MAX_NS], Ct = 0.f;
  for (int j = 0; j < P.ns; ++j) {
    Cw[j] = rw[j] * P.invM[j];
    Ct += Cw[j];
  }
  const float TK = P.T3T0 * Tw;
  for (int r = 0; r < P.nr; ++r) {
    const float k = P.k0[r] * expf(-P.EaR[r] / TK);
    if (P.rate_form[r] == FDLBM_RATE_CONC_BILINEAR) {
      float prod = 1.f;
      for (int j = 0; j < P.ns; ++j)
        for (int q = 0; q < -P.nu[r][j]; ++q) prod *= Cw[j];
      rate[r] = k * prod;
    } else {
      float fwd = 1.f, bwd = 1.f;
      for (int j = 0; j < P.ns; ++j) {
        const float xj = Cw[j] / Ct;
        for (int q = 0; q < -P.nu[r][j]; ++q) fwd *= xj;
        for (int q = 0; q < P.nu[r][j]; ++q) bwd *= xj;
      }
      rate[r] = k * (fwd - bwd * P.inv_Keq[r]);
    }
  }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;
}

constexpr int SOLID_BLOCK = 128;

__global__ void __launch_bounds__(SOLID_BLOCK) solid_kernel(DevParams P, const float* __restrict__ src,
                                                            float* __restrict__ dst,
                                                            const float* __restrict__ Ts_src,
                                                            float* __restrict__ Ts_dst,
                                                            const uint32_t* __restrict__ code,
                                                            const int32_t* __restrict__ list,
                                                            const float* __restrict__ Tgas,
                                                            double* __restrict__ ledger) {
  __shared__ double sh[SOLID_BLOCK / 32];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double acc_q = 0.0, acc_w = 0.0, acc_c = 0.0, acc_f = 0.0, acc_nc = 0.0;
  if (t < P.n_solid_list) {
    const int n = __ldg(list + t);
    const int x = n % P.nx, y = n / P.nx;
    const uint32_t cw = __ldg(code + n);
    const float Tx = Ts_src[n];
    float lap = 0.f, gas_term = 0.f;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int ox = d == 0 ? 1 : d == 1 ? -1 : 0;
      const int oy = d == 2 ? 1 : d == 3 ? -1 : 0;
      const int nb = lat_index(P, x + ox, y + oy);
      if (nb < 0) {
        const int face = d == 0 ? 1 : d == 1 ? 0 : d == 2 ? 3 : 2;
        if (P.fixedT_face[face]) {
          lap += P.dTout - Tx;
          acc_f += double(P.rhocp_s) * double(P.alpha_s) * double(P.dTout - Tx);
        }
        continue;
      }
      const uint32_t c = node_class(__ldg(code + nb));
      if (c == WALL || c == SOLID) lap += Ts_src[nb] - Tx;
      else if (c == GAS && Tgas != nullptr) gas_term += Tgas[nb] - (P.Tref + Tx);
    }
    float Tn = fmaf(P.alpha_s, lap, Tx);
    if (node_class(cw) == WALL) {
      const float Tw = P.Tref + Tx;
      // Arrival directions carry a stencil code; the wall emits along the opposite
      // directions (towards its gas neighbours).
      uint32_t arr = 0;
      float B = 0.f;
      for (int i = 1; i < Q; ++i)
        if (stencil_of(cw, i) != ST_NOT_ARRIVAL) arr |= 1u << i;
      for (int i = 1; i < Q; ++i)
        if (arr & (1u << OPP(i))) B += wrest(i, Tw);
      float A[MAX_NS], rw[MAX_NS], mj[MAX_NS];
      float Earr = 0.f;
      for (int j = 0; j < P.ns; ++j) {
        float a = 0.f;
        for (int i = 1; i < Q; ++i) {
          if (!(arr & (1u << i))) continue;
          const float v = pull_rt(P, src, j, i, x, y, n, stencil_of(cw, i)) + P.rref[j] * P.W0[i];
          a += v;
          Earr = fmaf(0.5f * P.c2[j] * float(EX(i) * EX(i) + EY(i) * EY(i)), v, Earr);
        }
        A[j] = a;
        rw[j] = a / B;
        mj[j] = 0.f;
      }
      float rate[MAX_NR] = {0.f, 0.f, 0.f, 0.f};
      const bool cat = (cw & CATALYTIC_BIT) && P.nr > 0;
      if (cat) {
        bool conv = false;
        for (int it = 0; it < P.rho_w_maxit; ++it) {
          rates(P, rw, Tw, rate);
          float d = 0.f, rmax = 0.f;
          for (int j = 0; j < P.ns; ++j) {
            float m = 0.f;
            for (int r = 0; r < P.nr; ++r) m += P.M[j] * float(P.nu[r][j]) * rate[r];
            const float nw = (A[j] + m) / B;
            d = fmaxf(d, fabsf(nw - rw[j]));
            rmax = fmaxf(rmax, fabsf(nw));
            rw[j] = nw;
          }
          if (d <= fmaxf(P.rho_w_tol, 4.f * FLT_EPSILON * rmax)) { conv = true; break; }
        }
        if (!conv) acc_nc += 1.0;
        rates(P, rw, Tw, rate);
        for (int j = 0; j < P.ns; ++j) {
          float m = 0.f;
          for (int r = 0; r < P.nr; ++r) m += P.M[j] * float(P.nu[r][j]) * rate[r];
          mj[j] = m;
        }
      }
      float Eout = 0.f;
      for (int j = 0; j < P.ns; ++j) {
        const float scale = (A[j] + mj[j]) / B;
        for (int i = 1; i < Q; ++i) {
          if (!(arr & (1u << OPP(i)))) continue;
          const float w = wrest(i, Tw) * scale;
          dst[(long long)(j * Q + i) * P.plane + n] = w - P.rref[j] * P.W0[i];
          Eout = fmaf(0.5f * P.c2[j] * float(EX(i) * EX(i) + EY(i) * EY(i)), w, Eout);
        }
      }
      float q = 0.f;
      if (cat)
        for (int r = 0; r < P.nr; ++r) q += P.heat[r] * rate[r];
      const float dE = Eout - Earr;
      const float couple = P.coupling == FDLBM_COUPLING_PAPER ? P.kappa_f * gas_term : -dE;
      Tn += (q + couple) * P.inv_rhocp_s;
      acc_q = q;
      acc_w = dE;
      acc_c = couple;
    }
    Ts_dst[n] = Tn;
  }
  // Block-reduce the FP64 ledger increments, one atomic per block and term.
  const double s_q = block_sum(acc_q, sh);
  const double s_w = block_sum(acc_w, sh);
  const double s_c = block_sum(acc_c, sh);
  const double s_f = block_sum(acc_f, sh);
  const double s_n = block_sum(acc_nc, sh);
  if (threadIdx.x == 0) {
    if (s_q != 0.0) atomicAdd(ledger + LG_QRXN, s_q);
    if (s_w != 0.0) atomicAdd(ledger + LG_QWALL, s_w);
    if (s_c != 0.0) atomicAdd(ledger + LG_QCOUPLE, s_c);
    if (s_f != 0.0) atomicAdd(ledger + LG_QFIXEDT, s_f);
    if (s_n != 0.0) atomicAdd(ledger + LG_NOCONV, s_n);
  }
}

// ---------------------------------------------------------------------------------------
// Initialisation (FP64 arithmetic, then rounded)
// ---------------------------------------------------------------------------------------
__device__ double wfac_d(int e, double v, double M, double T) {
  return e == 0 ? 1.0 - M * v * v - T : 0.5 * (double(e) * sqrt(M) * v + M * v * v + T);
}

__global__ void init_kernel(DevParams P, float* __restrict__ h0, float* __restrict__ h1,
                            float* __restrict__ Ts0, float* __restrict__ Ts1, float* __restrict__ mom,
                            float* __restrict__ Tgas, const uint32_t* __restrict__ code,
                            const double* __restrict__ X, const double* __restrict__ u,
                            const double* __restrict__ Tl, const double* __restrict__ Tsl,
                            const double* __restrict__ Cn, const double* __restrict__ inlet_u,
                            const double* __restrict__ X_inlet, double Tref) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P.n) return;
  const int x = n % P.nx, y = n / P.nx;
  const uint32_t c = node_class(code[n]);
  double Xn[MAX_NS];
  for (int j = 0; j < P.ns; ++j) Xn[j] = X[(long long)j * P.n + n];
  double ux = u[n], uy = u[P.n + n], T = Tl[n], C = Cn[n];
  if (c == INLET) {
    for (int j = 0; j < P.ns; ++j) Xn[j] = X_inlet[j];
    ux = inlet_u[y];
    uy = 0.0;
    T = X_inlet[P.ns];
    C = 1.0;
  }
  for (int j = 0; j < P.ns; ++j)
    for (int i = 0; i < Q; ++i) {
      h0[(long long)(j * Q + i) * P.plane + n] = 0.f;
      h1[(long long)(j * Q + i) * P.plane + n] = 0.f;
    }
  Ts0[n] = Ts1[n] = 0.f;
  if (c == GAS || c == INLET || c == OUTLET) {
    for (int j = 0; j < P.ns; ++j) {
      const double M = P.M[j];
      const double rho = C * Xn[j] * M;
      for (int i = 0; i < Q; ++i) {
        const double f = rho * wfac_d(EX(i), ux, M, T) * wfac_d(EY(i), uy, M, T);
        const double w0 = (EX(i) == 0 ? 1.0 - Tref : 0.5 * Tref) * (EY(i) == 0 ? 1.0 - Tref : 0.5 * Tref);
        const float v = float(f - double(P.rref[j]) * w0);
        h0[(long long)(j * Q + i) * P.plane + n] = v;
        h1[(long long)(j * Q + i) * P.plane + n] = v;
      }
    }
    if (c == GAS) {
      for (int j = 0; j < P.ns; ++j) mom[(long long)j * P.n + n] = float(C * Xn[j] * P.M[j]);
      mom[(long long)P.ns * P.n + n] = float(ux);
      mom[(long long)(P.ns + 1) * P.n + n] = float(uy);
      mom[(long long)(P.ns + 2) * P.n + n] = float(T);
      Tgas[n] = float(T);
    }
  } else if (c == WALL || c == SOLID) {
    const double Ts = Tsl[n];
    Ts0[n] = Ts1[n] = float(Ts - Tref);
    if (c == WALL) {
      const uint32_t cw = code[n];
      for (int j = 0; j < P.ns; ++j) {
        const double rho = C * Xn[j] * P.M[j];
        for (int i = 1; i < Q; ++i) {
          if (stencil_of(cw, OPP(i)) == ST_NOT_ARRIVAL) continue;
          const double wr = (EX(i) == 0 ? 1.0 - Ts : 0.5 * Ts) * (EY(i) == 0 ? 1.0 - Ts : 0.5 * Ts);
          const double w0 = (EX(i) == 0 ? 1.0 - Tref : 0.5 * Tref) * (EY(i) == 0 ? 1.0 - Tref : 0.5 * Tref);
          const float v = float(rho * wr - double(P.rref[j]) * w0);
          h0[(long long)(j * Q + i) * P.plane + n] = v;
          h1[(long long)(j * Q + i) * P.plane + n] = v;
        }
      }
    }
  }
  (void)x;
}

// ---------------------------------------------------------------------------------------
// Outputs and reductions
// ---------------------------------------------------------------------------------------
__global__ void moments_out_kernel(DevParams P, const float* __restrict__ mom, const float* __restrict__ Ts,
                                   const uint32_t* __restrict__ code, float* __restrict__ dst) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P.n) return;
  const int ns = P.ns;
  const uint32_t c = node_class(code[n]);
  const long long N = P.n;
  for (int f = 0; f < 2 * ns + 4; ++f) dst[f * N + n] = 0.f;
  if (c == GAS) {
    float C = 0.f;
    for (int j = 0; j < ns; ++j) C += mom[j * N + n] * P.invM[j];
    for (int j = 0; j < ns; ++j) {
      dst[j * N + n] = mom[j * N + n];
      dst[(ns + j) * N + n] = mom[j * N + n] * P.invM[j] / C;
    }
    dst[(2 * ns) * N + n] = mom[ns * N + n];
    dst[(2 * ns + 1) * N + n] = mom[(ns + 1) * N + n];
    dst[(2 * ns + 2) * N + n] = mom[(ns + 2) * N + n] * P.T3T0;
  } else if (c == WALL || c == SOLID) {
    dst[(2 * ns + 3) * N + n] = (P.Tref + Ts[n]) * P.T3T0;
  }
}

__global__ void populations_out_kernel(DevParams P, const float* __restrict__ h, float* __restrict__ dst) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)P.ns * Q * P.n;
  if (k >= total) return;
  const int n = int(k % P.n);
  const int ji = int(k / P.n);
  const int j = ji / Q, i = ji % Q;
  dst[k] = h[(long long)ji * P.plane + n] + P.rref[j] * P.W0[i];
}

// Ledger totals: E_gas (f-moments + in-transit wall emissions), H_solid, mass_j, moles_j.
__global__ void totals_kernel(DevParams P, const float* __restrict__ mom, const float* __restrict__ h,
                              const float* __restrict__ Ts, const uint32_t* __restrict__ code,
                              double* __restrict__ out) {
  __shared__ double sh[8];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int ns = P.ns;
  const long long N = P.n;
  double E = 0.0, H = 0.0, mass[MAX_NS], moles[MAX_NS];
  for (int j = 0; j < ns; ++j) mass[j] = moles[j] = 0.0;
  if (n < P.n) {
    const uint32_t cw = code[n];
    const uint32_t c = node_class(cw);
    if (c == GAS) {
      double C = 0.0, r = 0.0;
      for (int j = 0; j < ns; ++j) {
        const double rj = mom[j * N + n];
        mass[j] = rj;
        moles[j] = rj * double(P.invM[j]);
        C += rj / double(P.M[j]);
        r += rj;
      }
      const double ux = mom[ns * N + n], uy = mom[(ns + 1) * N + n], T = mom[(ns + 2) * N + n];
      E = C * T + 0.5 * r * (ux * ux + uy * uy);
    } else if (c == WALL || c == SOLID) {
      H = double(P.rhocp_s) * (double(P.Tref) + double(Ts[n]));
      if (c == WALL) {
        for (int i = 1; i < Q; ++i) {
          if (stencil_of(cw, OPP(i)) == ST_NOT_ARRIVAL) continue;
          for (int j = 0; j < ns; ++j) {
            const double w = double(h[(long long)(j * Q + i) * P.plane + n]) + double(P.rref[j]) * double(P.W0[i]);
            mass[j] += w;
            moles[j] += w / double(P.M[j]);
            E += 0.5 * double(P.c2[j]) * double(EX(i) * EX(i) + EY(i) * EY(i)) * w;
          }
        }
      }
    }
  }
  double s = block_sum(E, sh);
  if (threadIdx.x == 0) atomicAdd(out + 0, s);
  s = block_sum(H, sh);
  if (threadIdx.x == 0) atomicAdd(out + 1, s);
  for (int j = 0; j < ns; ++j) {
    s = block_sum(mass[j], sh);
    if (threadIdx.x == 0) atomicAdd(out + 2 + j, s);
    s = block_sum(moles[j], sh);
    if (threadIdx.x == 0) atomicAdd(out + 2 + ns + j, s);
  }
}

// Residual sums: for each field F (ux, uy, X_j, T on gas nodes; Ts on solid nodes):
// sum (F - snap)^2 and sum (F - ref)^2; then the snapshot is updated.
__global__ void residual_kernel(DevParams P, const float* __restrict__ mom, const float* __restrict__ Ts,
                                const uint32_t* __restrict__ code, float* __restrict__ snap,
                                double* __restrict__ out) {
  __shared__ double sh[8];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int ns = P.ns, nf = ns + 4;
  const long long N = P.n;
  float cur[MAX_NS + 4];
  bool on_gas = false, on_solid = false;
  if (n < P.n) {
    const uint32_t c = node_class(code[n]);
    on_gas = c == GAS;
    on_solid = c == WALL || c == SOLID;
    for (int f = 0; f < nf; ++f) cur[f] = 0.f;
    if (on_gas) {
      float C = 0.f;
      for (int j = 0; j < ns; ++j) C += mom[j * N + n] * P.invM[j];
      cur[0] = mom[ns * N + n];
      cur[1] = mom[(ns + 1) * N + n];
      for (int j = 0; j < ns; ++j) cur[2 + j] = mom[j * N + n] * P.invM[j] / C;
      cur[2 + ns] = mom[(ns + 2) * N + n];
    }
    if (on_solid) cur[3 + ns] = P.Tref + Ts[n];
  }
  for (int f = 0; f < nf; ++f) {
    const bool on = f == nf - 1 ? on_solid : on_gas;
    double dd = 0.0, dr = 0.0;
    if (on) {
      const double ref = f < 2 ? 0.0 : (f < 2 + ns ? double(P.Xin[f - 2]) : double(P.Tin_lat));
      const double a = cur[f], b = snap[f * N + n];
      dd = (a - b) * (a - b);
      dr = (a - ref) * (a - ref);
    }
    double s = block_sum(dd, sh);
    if (threadIdx.x == 0) atomicAdd(out + 2 * f, s);
    s = block_sum(dr, sh);
    if (threadIdx.x == 0) atomicAdd(out + 2 * f + 1, s);
  }
  if (n < P.n)
    for (int f = 0; f < nf; ++f) snap[f * N + n] = cur[f];
}

cudaError_t solid_ns(const DevParams& P, const DevState& S, int src, cudaStream_t st) {
  if (P.n_solid_list <= 0) return cudaSuccess;
  const int dstb = 1 - src;
  float* Tg = P.coupling == FDLBM_COUPLING_PAPER ? S.Tgas : nullptr;
  const int nb = (P.n_solid_list + SOLID_BLOCK - 1) / SOLID_BLOCK;
  solid_kernel<<<nb, SOLID_BLOCK, 0, st>>>(P, S.h[src], S.h[dstb], S.Ts[src], S.Ts[dstb], S.code, S.solid_list,
                                           Tg, S.ledger);
  return cudaGetLastError();
}

template <int NS>
cudaError_t gas_ns(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st) {
  const int dstb = 1 - src;
  dim3 block(TX, TY);
  dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
  float* Tg = P.coupling == FDLBM_COUPLING_PAPER ? S.Tgas : nullptr;
  if (moments_only) {
    if (P.energy_correction)
      gas_kernel<NS, true, 1><<<grid, block, 0, st>>>(P, S.h[src], S.h[dstb], S.code, S.mom, nullptr, S.flags);
    else
      gas_kernel<NS, false, 1><<<grid, block, 0, st>>>(P, S.h[src], S.h[dstb], S.code, S.mom, nullptr, S.flags);
  } else {
    if (P.energy_correction)
      gas_kernel<NS, true, 0><<<grid, block, 0, st>>>(P, S.h[src], S.h[dstb], S.code, nullptr, Tg, S.flags);
    else
      gas_kernel<NS, false, 0><<<grid, block, 0, st>>>(P, S.h[src], S.h[dstb], S.code, nullptr, Tg, S.flags);
  }
  return cudaGetLastError();
}

cudaError_t dispatch_gas(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st) {
  switch (P.ns) {
    case 1: return gas_ns<1>(P, S, src, moments_only, st);
    case 2: return gas_ns<2>(P, S, src, moments_only, st);
    case 3: return gas_ns<3>(P, S, src, moments_only, st);
    case 4: return gas_ns<4>(P, S, src, moments_only, st);
    case 5: return gas_ns<5>(P, S, src, moments_only, st);
    case 6: return gas_ns<6>(P, S, src, moments_only, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_init(const DevParams& P, const DevState& S, const double* X, const double* u,
                        const double* T_lat, const double* Ts_lat, const double* C, const double* inlet,
                        cudaStream_t st) {
  const double* X_inlet = inlet + P.ny;
  const int nb = (P.n + 255) / 256;
  init_kernel<<<nb, 256, 0, st>>>(P, S.h[0], S.h[1], S.Ts[0], S.Ts[1], S.mom, S.Tgas, S.code, X, u, T_lat, Ts_lat,
                                  C, inlet, X_inlet, double(P.Tref));
  return cudaGetLastError();
}

cudaError_t launch_step(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st) {
  if (moments_only) return dispatch_gas(P, S, src, true, st);
  cudaError_t e = solid_ns(P, S, src, st);
  if (e != cudaSuccess) return e;
  return dispatch_gas(P, S, src, false, st);
}

cudaError_t launch_solid(const DevParams& P, const DevState& S, int src, cudaStream_t st) {
  return solid_ns(P, S, src, st);
}

cudaError_t launch_gas(const DevParams& P, const DevState& S, int src, cudaStream_t st) {
  return dispatch_gas(P, S, src, false, st);
}

cudaError_t launch_moments_out(const DevParams& P, const DevState& S, int cur, float* dst, cudaStream_t st) {
  const int nb = (P.n + 255) / 256;
  moments_out_kernel<<<nb, 256, 0, st>>>(P, S.mom, S.Ts[cur], S.code, dst);
  return cudaGetLastError();
}

cudaError_t launch_populations_out(const DevParams& P, const DevState& S, int cur, float* dst, cudaStream_t st) {
  const long long total = (long long)P.ns * Q * P.n;
  const int nb = int((total + 255) / 256);
  populations_out_kernel<<<nb, 256, 0, st>>>(P, S.h[cur], dst);
  return cudaGetLastError();
}

cudaError_t launch_totals(const DevParams& P, const DevState& S, int cur, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(S.red, 0, sizeof(double) * totals_count(P.ns), st);
  if (e != cudaSuccess) return e;
  const int nb = (P.n + 255) / 256;
  totals_kernel<<<nb, 256, 0, st>>>(P, S.mom, S.h[cur], S.Ts[cur], S.code, S.red);
  return cudaGetLastError();
}

cudaError_t launch_residual(const DevParams& P, const DevState& S, int cur, cudaStream_t st) {
  double* out = S.red + totals_count(P.ns);
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * residual_count(P.ns), st);
  if (e != cudaSuccess) return e;
  const int nb = (P.n + 255) / 256;
  residual_kernel<<<nb, 256, 0, st>>>(P, S.mom, S.Ts[cur], S.code, S.snap, out);
  return cudaGetLastError();
}

}  // namespace fdlbm
