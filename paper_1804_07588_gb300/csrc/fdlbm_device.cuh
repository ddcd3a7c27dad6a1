// Device code of the solver that touches population storage, templated on the storage
// type PT of the populations: float (FP32), __nv_bfloat16 (BF16) or __half (FP16 with a
// per-species power-of-two scale). Included by the solver's kernel translation units:
// fdlbm_kernels.cu instantiates the FP32 path, fdlbm_store_bf16.cu and
// fdlbm_store_fp16.cu the 16-bit paths; each path runs the same FP32 arithmetic.
#pragma once

#include <cfloat>
#include <cmath>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fdlbm_internal.h"

namespace fdlbm {

namespace {

constexpr int GB = 256;  // gas kernel block size (threads = gas nodes)
// Resident blocks of the step kernel per SM: 3 caps it at 80 registers (with part of the
// pulled values in shared memory, see NSC_OF) and runs 24 warps per SM: on the 1024x512 bed
// 10% faster than 2 blocks at 128 registers; 4 blocks (64 registers) spill and lose.
#ifndef GAS_MIN_BLOCKS
#define GAS_MIN_BLOCKS 3
#endif

__host__ __device__ constexpr int EX(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0; }
__host__ __device__ constexpr int EY(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0; }
__host__ __device__ constexpr int OPP(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5); }
// Forcing coefficients of Eq. psi_jialpha times 4 c_j.
__host__ __device__ constexpr float PSX(int i) { return i == 1 ? 4.f : i == 3 ? -4.f : (i == 5 || i == 8) ? -1.f : (i == 6 || i == 7) ? 1.f : 0.f; }
__host__ __device__ constexpr float PSY(int i) { return i == 2 ? 4.f : i == 4 ? -4.f : (i == 5 || i == 6) ? -1.f : (i == 7 || i == 8) ? 1.f : 0.f; }

__device__ __forceinline__ int pad_index(const DevParams& P, int x, int y) {
  return (x + P.xoff) + (y + P.yoff) * P.pitch;
}

// Compact index of (x, y) wrapped on periodic axes; -1 off the lattice.
__device__ __forceinline__ int lat_index(const DevParams& P, int x, int y) {
  if (x < 0) { if (!P.periodic_x) return -1; x += P.nx; }
  else if (x >= P.nx) { if (!P.periodic_x) return -1; x -= P.nx; }
  if (y < 0) { if (!P.periodic_y) return -1; y += P.ny; }
  else if (y >= P.ny) { if (!P.periodic_y) return -1; y -= P.ny; }
  return x + P.nx * y;
}

// Padded-lattice offsets of the ghost copies a node at (x, y) must also write: along x
// and y (0 when none) on periodic axes within GHOST of a face.
struct Ghost { int dx, dy; };
__device__ __forceinline__ Ghost ghost_of(const DevParams& P, int x, int y) {
  Ghost g{0, 0};
  if (P.periodic_x) g.dx = x < GHOST ? P.nx : (x >= P.nx - GHOST ? -P.nx : 0);
  if (P.periodic_y) g.dy = y < GHOST ? P.ny * P.pitch : (y >= P.ny - GHOST ? -P.ny * P.pitch : 0);
  return g;
}
// Populations are written once per step and read only by the next step: streaming
// (evict-first) stores keep L2 for the current step's reads.
__device__ __forceinline__ void store_with_ghosts(float* p, int k, const Ghost& g, float v) {
  __stcs(p + k, v);
  if (g.dx) __stcs(p + k + g.dx, v);
  if (g.dy) {
    __stcs(p + k + g.dy, v);
    if (g.dx) __stcs(p + k + g.dx + g.dy, v);
  }
}

// Population storage. PT is float (FP32), __nv_bfloat16 or __half; every value is the
// deviation h = g - rref_j W0_i, the __half form scaled by a power of two per species
// (P.hs[j]; P.hsi[j] is its inverse) so that the deviations sit inside FP16's range.
// Arithmetic is FP32 throughout; values are rounded to T once, when stored.
__device__ __forceinline__ float pop_ld(const float* p, float) { return __ldg(p); }
__device__ __forceinline__ float pop_ld(const __nv_bfloat16* p, float) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float pop_ld(const __half* p, float inv) { return __half2float(__ldg(p)) * inv; }
template <class PT> __device__ __forceinline__ PT pop_enc(float v, float sc);
template <> __device__ __forceinline__ float pop_enc<float>(float v, float) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 pop_enc<__nv_bfloat16>(float v, float) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half pop_enc<__half>(float v, float sc) { return __float2half_rn(v * sc); }
// Streaming (evict-first) store of an encoded value.
__device__ __forceinline__ void pop_stcs(float* p, float e) { __stcs(p, e); }
__device__ __forceinline__ void pop_stcs(__nv_bfloat16* p, __nv_bfloat16 e) {
  __stcs(reinterpret_cast<unsigned short*>(p), __bfloat16_as_ushort(e));
}
__device__ __forceinline__ void pop_stcs(__half* p, __half e) {
  __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(e));
}
// Stores made by the time step round the 16-bit forms stochastically: random low bits are
// added to the FP32 bit pattern of the (scaled) value before truncation, so that a value
// rounds up with probability equal to its distance from the lower neighbour. The mean
// stored value is the exact one: a nearly steady population does not get the same
// rounding error every step (round-to-nearest would act as a persistent mass and momentum
// source). The random bits come from a counter-based hash of (node, population, step),
// so runs are reproducible. FP16 values below 2^-14 after scaling (more than 13 dropped
// bits) round towards zero slightly more often.
__device__ __forceinline__ uint32_t hash32(uint32_t x) {  // "lowbias32" integer hash (C. Wellons)
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ uint32_t node_seed(int k, uint32_t step) { return hash32(uint32_t(k) * 0x9E3779B9U + hash32(step)); }
__device__ __forceinline__ uint32_t pop_random(uint32_t seed, int q) { return hash32(seed ^ (uint32_t(q) * 0x85EBCA6BU)); }
template <class PT> __device__ __forceinline__ PT pop_round(float v, float sc, uint32_t r);
template <> __device__ __forceinline__ float pop_round<float>(float v, float, uint32_t) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 pop_round<__nv_bfloat16>(float v, float, uint32_t r) {
  return __ushort_as_bfloat16((unsigned short)((__float_as_uint(v) + (r & 0xFFFFU)) >> 16));
}
template <> __device__ __forceinline__ __half pop_round<__half>(float v, float sc, uint32_t r) {
  return __float2half_rz(__uint_as_float(__float_as_uint(v * sc) + (r & 0x1FFFU)));
}
template <class PT>
__device__ __forceinline__ void pop_put_ghosts(PT* p, int k, const Ghost& g, PT e) {
  pop_stcs(p + k, e);
  if (g.dx) pop_stcs(p + k + g.dx, e);
  if (g.dy) {
    pop_stcs(p + k + g.dy, e);
    if (g.dx) pop_stcs(p + k + g.dx + g.dy, e);
  }
}
// Store of a time-step result v of population q of a node with random seed `seed`.
template <class PT>
__device__ __forceinline__ void pop_store_ghosts(PT* p, int k, const Ghost& g, float v, float sc, uint32_t seed, int q) {
  pop_put_ghosts(p, k, g, pop_round<PT>(v, sc, sizeof(PT) == 4 ? 0U : pop_random(seed, q)));
}

// Species whose pulled values a gas-tile thread keeps in shared memory rather than registers
// (the last three, or all of them for NS <= 3): with the other pulled values and the
// collision's temporaries the kernel then fits 80 registers without spills (three blocks per
// SM; 43 KB of shared memory per block for 5 species).
template <int NS>
constexpr int NSC_OF = NS > 3 ? 3 : NS;

// Running species moments of pulled deviations.
template <int NS>
struct Acc {
  float dr[NS], ax[NS], ay[NS], e[NS];
};

// Exact-account increments of one gas node, FP64 sums of exact differences of FP32
// values (kept only by the exact-accounts step): energy taken from / lost into inlet and
// outlet nodes, the pulls' departure from the pure shift, the collision's change.
struct Acct {
  double qin, qout, dint, dcol;
};
// Energy weight (1/2) c_j^2 |e_i|^2 of population (j, i), exact in FP32.
__device__ __forceinline__ double eps_weight(const DevParams& P, int j, int e2) {
  return double(0.5f * P.c2[j] * float(e2));
}

// Branch-free form of every streaming stencil: with s1 streamed from x - e_i and two more
// sources sA, sB at x + mA e_i and x + mB e_i, the pulled value is
//   s1 + (a/2) [(pA sA + pB sB) - (pA + pB) s1] + (a^2/2) [(qA sA + qB sB) - (qA + qB) s1]
// (a = 1 - c_j): central (Eq. interpol_bulk) sA = s2, sB = s0; forward (Eq.
// interpol_away) sA = s0, sB = s+; backward (Eq. interpol_towards) sA = s2, sB = s3;
// linear and none as degenerate cases. The brackets vanish exactly on uniform data.
struct StencilCoef {
  int mA, mB;
  float pA, pB, p1, qA, qB, q1;
};
__device__ __forceinline__ StencilCoef stencil_coef(uint32_t st) {
  StencilCoef c;
  const bool cen = st == ST_CENTRAL, fwd = st == ST_FORWARD, bwd = st == ST_BACKWARD;
  const bool l0 = st == ST_LIN_S0, l2 = st == ST_LIN_S2;
  c.mA = (cen || bwd || l2) ? -2 : 0;
  c.mB = fwd ? 1 : (bwd ? -3 : (l2 ? -2 : 0));
  c.pA = cen ? -1.f : fwd ? 4.f : bwd ? -4.f : l0 ? 2.f : l2 ? -2.f : 0.f;
  c.pB = cen ? 1.f : fwd ? -1.f : bwd ? 1.f : 0.f;
  c.p1 = cen ? 0.f : fwd ? 3.f : bwd ? -3.f : l0 ? 2.f : l2 ? -2.f : 0.f;
  c.qA = cen ? 1.f : (fwd || bwd) ? -2.f : 0.f;
  c.qB = (cen || fwd || bwd) ? 1.f : 0.f;
  c.q1 = cen ? 2.f : (fwd || bwd) ? -1.f : 0.f;
  return c;
}

// Streaming stencil coefficients by stencil code (the values of stencil_coef): {pA, pB,
// p1, qA}, {qB, q1} and the integer offsets {mA, mB} in units of e_i.
__constant__ float4 c_st_p[8] = {{0.f, 0.f, 0.f, 0.f},   {-1.f, 1.f, 0.f, 1.f}, {4.f, -1.f, 3.f, -2.f},
                                 {-4.f, 1.f, -3.f, -2.f}, {2.f, 0.f, 2.f, 0.f},  {-2.f, 0.f, -2.f, 0.f},
                                 {0.f, 0.f, 0.f, 0.f},    {0.f, 0.f, 0.f, 0.f}};
__constant__ float2 c_st_q[8] = {{0.f, 0.f}, {1.f, 2.f}, {1.f, -1.f}, {1.f, -1.f},
                                 {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f},  {0.f, 0.f}};
__constant__ int2 c_st_m[8] = {{0, 0}, {-2, 0}, {0, 1}, {-2, -3}, {0, 0}, {-2, -2}, {0, 0}, {0, 0}};

// Pull direction I of every species into the gas node at padded index k: the upstream
// value s1 = h_I(x - e_I) and, for off-lattice species, the two further stencil points,
// all loads of the direction issued together; the interpolated value goes to the
// thread's register array hv[j Q + I] and into the moment accumulators. DET: the exact
// accounts of the pull (departure from the shift, inlet/outlet face fluxes).
template <class PT, int NS, int I, bool DET>
__device__ __forceinline__ void pull_dir(const DevParams& P, const PT* __restrict__ src,
                                         const uint32_t* __restrict__ code, int k, uint32_t cw, Acc<NS>& a,
                                         float (&hv)[NS * Q], float* __restrict__ scol, const float (&ecoef)[3],
                                         Acct* ac) {
  constexpr int e2 = EX(I) * EX(I) + EY(I) * EY(I);
  if (I == 0) {
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const float v = pop_ld(src + ((j * Q) * (int)P.plane + k), P.hsi[j]);
      if (j >= NS - NSC_OF<NS>) scol[(j - (NS - NSC_OF<NS>)) * Q * GB] = v;
      else hv[j * Q] = v;
      a.dr[j] += v;
      a.e[j] = fmaf(ecoef[0], v, a.e[j]);
    }
    return;
  }
  const int off = EX(I) + EY(I) * P.pitch;
  // exact accounts: classes of the upstream node (source of s1) and of the node this
  // node's own population I streams into
  uint32_t cu = GAS, cd = GAS;
  if constexpr (DET) {
    cu = node_class(__ldg(code + k - off));
    cd = node_class(__ldg(code + k + off));
  }
  const uint32_t st = stencil_of(cw, I);
  const float4 cp = c_st_p[st];
  const float2 cq = c_st_q[st];
  const int2 cm = c_st_m[st];
  const int dA = cm.x * off, dB = cm.y * off;
  float v1[NS], vA[NS], vB[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const int b = (j * Q + I) * (int)P.plane + k;
    v1[j] = pop_ld(src + (b - off), P.hsi[j]);
    vA[j] = vB[j] = 0.f;
    if (!P.onlattice[j]) {
      vA[j] = pop_ld(src + (b + dA), P.hsi[j]);
      vB[j] = pop_ld(src + (b + dB), P.hsi[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    float v = v1[j];
    if (!P.onlattice[j]) {
      const float d1 = fmaf(-cp.z, v1[j], fmaf(cp.x, vA[j], cp.y * vB[j]));
      const float d2 = fmaf(-cq.y, v1[j], fmaf(cp.w, vA[j], cq.x * vB[j]));
      v = fmaf(P.ha[j], d1, fmaf(P.ha2[j], d2, v1[j]));
    }
    if constexpr (DET) {
      const double e = eps_weight(P, j, e2);
      ac->dint += e * (double(v) - double(v1[j]));
      const double off0 = double(P.rref[j]) * double(P.W0[I]);
      if (cu == INLET) ac->qin += e * (double(v1[j]) + off0);
      if (cu == OUTLET) ac->qout += e * (double(v1[j]) + off0);
      if (cd == INLET || cd == OUTLET) {
        const double own = e * (double(pop_ld(src + ((j * Q + I) * (int)P.plane + k), P.hsi[j])) + off0);
        if (cd == INLET) ac->qin -= own;
        else ac->qout -= own;
      }
    }
    if (j >= NS - NSC_OF<NS>) scol[((j - (NS - NSC_OF<NS>)) * Q + I) * GB] = v;
    else hv[j * Q + I] = v;
    a.dr[j] += v;
    if (EX(I) > 0) a.ax[j] += v;
    if (EX(I) < 0) a.ax[j] -= v;
    if (EY(I) > 0) a.ay[j] += v;
    if (EY(I) < 0) a.ay[j] -= v;
    a.e[j] = fmaf(ecoef[e2], v, a.e[j]);
  }
}

// Stream all populations into the gas node at padded index k (pull streaming with the
// off-lattice interpolation of Sec. 4.2) and accumulate the species moments.
template <class PT, int NS, bool DET>
__device__ __forceinline__ void pull_node(const DevParams& P, const PT* __restrict__ src,
                                          const uint32_t* __restrict__ code, int k, uint32_t cw, Acc<NS>& a,
                                          float (&hv)[NS * Q], float* __restrict__ scol, Acct* ac) {
  const float ecoef[3] = {-2.f * P.Tref, 1.f - 2.f * P.Tref, 2.f - 2.f * P.Tref};
#pragma unroll
  for (int j = 0; j < NS; ++j) a.dr[j] = a.ax[j] = a.ay[j] = a.e[j] = 0.f;
  pull_dir<PT, NS, 0, DET>(P, src, code, k, cw, a, hv, scol, ecoef, ac);
  pull_dir<PT, NS, 1, DET>(P, src, code, k, cw, a, hv, scol, ecoef, ac);
  pull_dir<PT, NS, 2, DET>(P, src, code, k, cw, a, hv, scol, ecoef, ac);
  pull_dir<PT, NS, 3, DET>(P, src, code, k, cw, a, hv, scol, ecoef, ac);
  pull_dir<PT, NS, 4, DET>(P, src, code, k, cw, a, hv, scol, ecoef, ac);
  pull_dir<PT, NS, 5, DET>(P, src, code, k, cw, a, hv, scol, ecoef, ac);
  pull_dir<PT, NS, 6, DET>(P, src, code, k, cw, a, hv, scol, ecoef, ac);
  pull_dir<PT, NS, 7, DET>(P, src, code, k, cw, a, hv, scol, ecoef, ac);
  pull_dir<PT, NS, 8, DET>(P, src, code, k, cw, a, hv, scol, ecoef, ac);
}

// Mixture moments from the species accumulators (Eq. moments_of_g, Eq. moments_of_f):
// densities, momenta, C and the g-temperature deviation dTg = T_g - T_ref.
template <int NS>
struct Mom {
  float drho[NS], Jx[NS], Jy[NS];
  float r, jx, jy, C, dTg;
};

template <int NS>
__device__ __forceinline__ void finish_moments(const DevParams& P, const Acc<NS>& a, Mom<NS>& m) {
  m.r = m.jx = m.jy = m.C = 0.f;
  float de = 0.f;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    m.drho[j] = a.dr[j];
    const float rho = P.rref[j] + a.dr[j];
    m.Jx[j] = P.c[j] * a.ax[j];
    m.Jy[j] = P.c[j] * a.ay[j];
    m.r += rho;
    m.jx += m.Jx[j];
    m.jy += m.Jy[j];
    m.C = fmaf(rho, P.invM[j], m.C);
    de = fmaf(P.c2[j], a.e[j], de);
  }
  m.dTg = (de - fmaf(m.jx, m.jx, m.jy * m.jy) / m.r) * (0.5f / m.C);
}

// One axis of the product-form equilibrium (Eq. eq_state_pop, positive-sign form) for
// velocity component v: factors w(e) and their deviations dw(e) from the rest factors
// at T_ref, index e + 1.
struct Axis {
  float w[3], dw[3];
};
__device__ __forceinline__ Axis axis_factors(float sqrtM, float sMlo, float M, float v, float T, float dT) {
  const float s = fmaf(sqrtM, v, sMlo * v), m = M * v * v;
  Axis a;
  a.w[1] = 1.f - m - T;
  a.w[2] = 0.5f * (m + T + s);
  a.w[0] = 0.5f * (m + T - s);
  a.dw[1] = -(m + dT);
  a.dw[2] = 0.5f * (m + dT + s);
  a.dw[0] = 0.5f * (m + dT - s);
  return a;
}

template <int NS>
__device__ __forceinline__ void flag_bad(int* flags, const Mom<NS>& m, float T) {
  if (!(m.r > 0.f) || !(T > 0.f) || !isfinite(m.jx + m.jy + T)) atomicOr(flags, 1);
}

// ---------------------------------------------------------------------------------------
// Gas tiles
// ---------------------------------------------------------------------------------------
// A gas block is a tile: the gas nodes of a band of rows and a range of columns (its
// interior, row-major), followed by the gas nodes of the one-node ring around it that
// are axis neighbours of interior gas nodes (its halo). Descriptor {role 0, first list
// entry, interior count << 16 | total count, map row stride}; gas_slot holds each
// entry's position in the tile's moment map (row stride Wp, the ring at the edges).
//
// Phase 1, every entry: pull streaming with the off-lattice interpolation (Sec. 4.2) into
// the thread's shared-memory column, moments (Eq. moments_of_g), and T_g and
// K_j = kcoef_j C_j T_g into the map. Phase 2, after a block barrier, interior entries
// only: divergence of the energy-correction flux K_j grad T_g on the 4 axis neighbours
// from the map, i.e. from the moments of the current time level (reading R8), the
// two-step collision (Eq. final_kinetic_equation), the outlet equilibrium and the
// streaming stores.
// MODE 0: full step. MODE 1: moments only (the pre-collision moments of the step that
// reads src into mom[] at compact indices; nothing else is written).
// LT: relaxation times updated per node from its pulled densities and g-temperature
// (Sec. 3, Eqs. tau1s with Wilke's rule, tau2_approx_text, D_j_text); they also enter
// K_j.

template <class PT, int NS, bool PHI, int MODE, bool LT = false, bool DET = false>
__device__ __forceinline__ void gas_tile(const DevParams& P, const PT* __restrict__ src, PT* __restrict__ dst,
                                         const uint32_t* __restrict__ code, const int2* __restrict__ gas_list,
                                         const uint16_t* __restrict__ gas_slot, const int4 d,
                                         float* __restrict__ mom, float* __restrict__ Tgas, int* __restrict__ flags,
                                         float* __restrict__ smem, uint32_t step, Acct* ac = nullptr) {
  const int tid = threadIdx.x;
  const int n_tot = d.z & 0xFFFF, n_int = d.z >> 16, Wp = d.w;
  float* s_map = smem;  // [1 + NS][GAS_MAP_SLOTS]: dTg, K_j of the tile and its halo
  uint32_t cw = 0;
  int k = 0, aux = 0, slot = 0;
  Acc<NS> acc;
  Mom<NS> m;
  float t1l[NS], t2l[NS];
  float hv[NS * Q];  // the pulled populations, in registers until the collision
  // ... except those of the last NSC_OF<NS> species, in the thread's column of shared memory
  // (stride GB)
  float* s_col = smem + (1 + NS) * GAS_MAP_SLOTS + tid;
  if (tid < n_tot) {
    const int2 g = __ldg(gas_list + d.y + tid);
    k = g.x;
    aux = g.y;
    if (PHI) slot = __ldg(gas_slot + d.y + tid);
    cw = __ldg(code + k);
    Acct halo_acct{0.0, 0.0, 0.0, 0.0};  // halo entries are counted by their own tile
    pull_node<PT, NS, DET>(P, src, code, k, cw, acc, hv, s_col, tid < n_int ? ac : &halo_acct);
    finish_moments<NS>(P, acc, m);
    // Local relaxation times: tau1_j = mu_j / (C T sum_k X_k phi_jk), tau2_j = rho_j D_j /
    // (X_j C T) = M_j (1 - Y_j) / (T sum_{k != j} X_k / D_jk), T the g-temperature.
    if constexpr (LT) {
      const float Tg = P.Tref + m.dTg;
      const float iC = 1.f / m.C;
      float X[NS];
#pragma unroll
      for (int j = 0; j < NS; ++j) X[j] = (P.rref[j] + m.drho[j]) * P.invM[j] * iC;
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        float sphi = 0.f, sd = 0.f;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          sphi = fmaf(X[q], P.phi_w[j][q], sphi);
          sd = fmaf(X[q], P.invD[j][q], sd);
        }
        t1l[j] = P.mu_l[j] / (m.C * Tg * sphi);
        t2l[j] = P.M[j] * (1.f - (P.rref[j] + m.drho[j]) / m.r) / (Tg * sd);
      }
    }
    if (PHI) {
      s_map[slot] = m.dTg;
#pragma unroll
      for (int j = 0; j < NS; ++j)
        s_map[(1 + j) * GAS_MAP_SLOTS + slot] = (LT ? P.kcoef0[j] * t1l[j] : P.kcoef[j]) *
                                                ((P.rref[j] + m.drho[j]) * P.invM[j]) * (P.Tref + m.dTg);
    }
  }
  if (PHI) __syncthreads();
  if (tid >= n_int) return;
  const int n = aux & GAS_AUX_N;
  const uint32_t seed = sizeof(PT) == 4 ? 0U : node_seed(k, step);

  // Divergence of the energy-correction flux K_j grad T on the 4 axis neighbours (+x, +y,
  // -x, -y: map slots +1, +Wp, -1, -Wp); faces to non-gas nodes carry no flux.
  float divq[NS];
  float sdq = 0.f;
#pragma unroll
  for (int j = 0; j < NS; ++j) divq[j] = 0.f;
  if (PHI) {
    const float Tc = s_map[slot];
    float Kc[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) Kc[j] = s_map[(1 + j) * GAS_MAP_SLOTS + slot];
#pragma unroll
    for (int dd = 1; dd <= 4; ++dd) {
      if (!((cw >> (NBR_GAS_SHIFT + dd - 1)) & 1u)) continue;
      const int sn = slot + (dd == 1 ? 1 : dd == 2 ? Wp : dd == 3 ? -1 : -Wp);
      const float dTn = s_map[sn] - Tc;
#pragma unroll
      for (int j = 0; j < NS; ++j) divq[j] = fmaf(0.5f * (Kc[j] + s_map[(1 + j) * GAS_MAP_SLOTS + sn]), dTn, divq[j]);
    }
#pragma unroll
    for (int j = 0; j < NS; ++j) sdq += divq[j];
  }

  const float ux = m.jx / m.r, uy = m.jy / m.r;
  const float dT = m.dTg + sdq / (4.f * m.C);
  const float T = P.Tref + dT;
  if (MODE == 1) {
#pragma unroll
    for (int j = 0; j < NS; ++j) mom[(long long)j * P.n + n] = P.rref[j] + m.drho[j];
    mom[(long long)NS * P.n + n] = ux;
    mom[(long long)(NS + 1) * P.n + n] = uy;
    mom[(long long)(NS + 2) * P.n + n] = dT;  // T - T_ref
    return;
  }
  Ghost gh{0, 0};
  if (aux & GAS_AUX_GHOST) gh = ghost_of(P, n % P.nx, n / P.nx);
  if (Tgas != nullptr) Tgas[n] = dT;  // T - T_ref
  flag_bad<NS>(flags, m, T);

  // Corrective diffusion velocity (reading R3: weights 1/(tau2 + 1/2)).
  float ncx = 0.f, ncy = 0.f, den = 0.f;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const float rho = P.rref[j] + m.drho[j];
    const float w = LT ? 1.f / (t2l[j] + 0.5f) : P.uc_w[j];
    ncx = fmaf(w, fmaf(-rho, ux, m.Jx[j]), ncx);
    ncy = fmaf(w, fmaf(-rho, uy, m.Jy[j]), ncy);
    den = fmaf(w, rho, den);
  }
  const float iden = 1.f / den;
  const float Ucx = ncx * iden, Ucy = ncy * iden;

  // Collision species by species; the species' density and momentum are the pull's sums.
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    float h[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i)
      h[i] = j >= NS - NSC_OF<NS> ? s_col[((j - (NS - NSC_OF<NS>)) * Q + i) * GB] : hv[j * Q + i];
    const float drj = m.drho[j];
    const float Jxj = m.Jx[j], Jyj = m.Jy[j], dqj = divq[j];
    const float rho = P.rref[j] + drj;
    // f-momentum of the species (Eq. moments_of_g) and its velocity, limited for trace
    // species (reading R15).
    // collision coefficients: per species constants, or from the node's relaxation times
    float a2j = P.a2[j], inv1a2j = P.inv1a2[j], omj = P.omega[j], omtj = P.omega[j] * P.t1t2[j];
    float wt1j = P.wt1[j], invtau2j = P.invtau2[j];
    if constexpr (LT) {
      const float t1 = t1l[j], t2 = t2l[j];
      omj = 2.f / (1.f + 2.f * t1);
      wt1j = omj * t1;
      invtau2j = 1.f / t2;
      omtj = wt1j * invtau2j;
      a2j = 0.5f * invtau2j;
      inv1a2j = 1.f / (1.f + a2j);
    }
    // Velocity of f*: u_j = (J_j + a2 rho_j (u + U^c)) / ((1 + a2) rho_j), formed as
    // u + (D_j + a2 rho_j U^c) / ((1 + a2) rho_j) from the diffusion flux D_j = J_j - rho_j u.
    // With the rounded constants a2, 1 / (1 + a2), omega, omega tau1 / tau2 the direct form
    // leaves a momentum source (B - A) rho_j u per collision, B - A ~ 1e-7 (the two
    // coefficients are equal in exact arithmetic), which builds up a velocity error
    // proportional to u over the steps; in this form no constant multiplies rho_j u.
    const float a2r = a2j * rho;
    float ujx = ux, ujy = uy;
    if (rho != 0.f) {
      const float ir = 1.f / rho;
      ujx = fmaf(fmaf(a2r, Ucx, fmaf(-rho, ux, Jxj)) * inv1a2j, ir, ux);
      ujy = fmaf(fmaf(a2r, Ucy, fmaf(-rho, uy, Jyj)) * inv1a2j, ir, uy);
      const float lim2 = fmaxf(1.f - T, 0.f) * P.invM[j];
      if (ujx * ujx > lim2 || ujy * ujy > lim2) {  // rare: trace species driven through zero
        const float lim = sqrtf(lim2);
        ujx = fminf(fmaxf(ujx, -lim), lim);
        ujy = fminf(fmaxf(ujy, -lim), lim);
      }
    }
    const float M = P.M[j], sM = P.sqrtM[j], sl = P.sqrtM_lo[j], dr = drj, rr = P.rref[j];
    const Axis ex = axis_factors(sM, sl, M, ux, T, dT), ey = axis_factors(sM, sl, M, uy, T, dT);
    const Axis sx = axis_factors(sM, sl, M, ujx, T, dT), sy = axis_factors(sM, sl, M, ujy, T, dT);
    // The deviation of rho wx(a) wy(b) from rref w0(a) w0(b), with p(a) = rho wx(a) -
    // rref w0(a) = drho w0(a) + rho dwx(a):  f(a, b) = p(a) w0(b) + (p(a) + rref w0(a)) dwy(b).
    // Only the rest factors w0 and the deviations dw (formed from T - T_ref) appear: the
    // factors w at the absolute temperature carry its rounding (~1.5e-8, nearly the same
    // on all nodes of a uniform region), which multiplied by drho would act as a
    // systematic energy source at every collision.
    const float w0e[3] = {0.5f * P.Tref, 1.f - P.Tref, 0.5f * P.Tref};
    float pe[3], ps[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      pe[e] = fmaf(dr, w0e[e], rho * ex.dw[e]);
      ps[e] = fmaf(dr, w0e[e], rho * sx.dw[e]);
    }
    const float q0 = rr * (1.f - P.Tref), q1 = rr * 0.5f * P.Tref;  // rref w0(0), rref w0(+-1)
    const float om = omj, omt = omtj;
    // w1 tau1 Psi_i = PSX_i gfx + PSY_i gfy with psi = PSX / (4 c_j), 1 / c_j = sqrt(M_j)
    const float gfs = wt1j * rho * invtau2j * 0.25f * P.sqrtM[j];
    const float gfx = gfs * Ucx, gfy = gfs * Ucy;
    // w1 tau1 Phi_i with phi = M_j {-1, 1/4 on the axis links, 0 on diagonals}
    const float gphi = wt1j * M * dqj;
    float hn[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int a = EX(i) + 1, b = EY(i) + 1;
      const float qa = EX(i) == 0 ? q0 : q1;
      const float feq = fmaf(pe[a], w0e[b], (pe[a] + qa) * ey.dw[b]);
      const float fst = fmaf(ps[a], w0e[b], (ps[a] + qa) * sy.dw[b]);
      float force = PSX(i) * gfx + PSY(i) * gfy;  // coefficients 0, +-1, +-4: no rounding choice
      if (i == 0) force -= gphi;
      else if (i <= 4) force = fmaf(0.25f, gphi, force);
      // h' = h - w1 (h - f*) - w1 (tau1 / tau2)(f* - f^eq) + w1 tau1 (Psi + Phi); the two
      // small differences are formed first so that FP32 keeps their precision.
      hn[i] = fmaf(-om, h[i] - fst, fmaf(-omt, fst - feq, h[i] + force));
    }
    if constexpr (DET) {  // FP32 storage: hn is the value stored
      double dc = 0.0;
#pragma unroll
      for (int i = 1; i < Q; ++i) dc += eps_weight(P, j, EX(i) * EX(i) + EY(i) * EY(i)) * (double(hn[i]) - double(h[i]));
      ac->dcol += dc;
    }
    // 32-bit element offsets: the host keeps ns Q plane below 2^31.
    const int pl = (int)P.plane;
    PT* out = dst + j * Q * pl;
    const float sc = P.hs[j];
    if (!(aux & GAS_AUX_GHOST)) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        pop_stcs(out + (i * pl + k), pop_round<PT>(hn[i], sc, sizeof(PT) == 4 ? 0U : pop_random(seed, j * Q + i)));
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) pop_store_ghosts(out + i * pl, k, gh, hn[i], sc, seed, j * Q + i);
    }
  }

  // Outlet (reading R13): equilibrium at the outlet pressure with this node's
  // composition, velocity and temperature.
  if (aux & GAS_AUX_OUTLET) {
    const float Cout = P.p_out / T;
    Ghost go{0, 0};
    if (aux & GAS_AUX_GHOST) go = ghost_of(P, n % P.nx + 1, n / P.nx);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const float rj = (P.rref[j] + m.drho[j]) * P.invM[j] / m.C * Cout * P.M[j];
      const float dr = rj - P.rref[j], rr = P.rref[j];
      const Axis ex = axis_factors(P.sqrtM[j], P.sqrtM_lo[j], P.M[j], ux, T, dT),
                 ey = axis_factors(P.sqrtM[j], P.sqrtM_lo[j], P.M[j], uy, T, dT);
      const float q0 = rr * (1.f - P.Tref), q1 = rr * 0.5f * P.Tref;
      const float w0e[3] = {0.5f * P.Tref, 1.f - P.Tref, 0.5f * P.Tref};
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int a = EX(i) + 1, b = EY(i) + 1;
        const float pa = fmaf(dr, w0e[a], rj * ex.dw[a]);
        const float v = fmaf(pa, w0e[b], (pa + (EX(i) == 0 ? q0 : q1)) * ey.dw[b]);
        pop_store_ghosts(dst + (long long)(j * Q + i) * P.plane, k + 1, go, v, P.hs[j], seed, NS * Q + j * Q + i);
      }
    }
  }
}

template <int NS, bool LT = false>
size_t gas_smem_bytes() {
  return sizeof(float) * ((1 + NS) * GAS_MAP_SLOTS + NSC_OF<NS> * Q * GB);  // moment map + the shared species' column
}

// ---------------------------------------------------------------------------------------
// Wall + solid kernel
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float wrest(int i, float T) {
  return (EX(i) == 0 ? 1.f - T : 0.5f * T) * (EY(i) == 0 ? 1.f - T : 0.5f * T);
}

// Reaction rates (lattice moles per wall node per step) at wall densities rw, with the
// Arrhenius factors k_r = k0_r exp(-Ea_r / (R T_w)) precomputed for this wall node.
template <int NS>
__device__ __forceinline__ void rates(const DevParams& P, const float (&rw)[NS], const float* kr, float* rate) {
  float Cw[NS], Ct = 0.f;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    Cw[j] = rw[j] * P.invM[j];
    Ct += Cw[j];
  }
  const float iCt = 1.f / Ct;
  for (int r = 0; r < P.nr; ++r) {
    float fwd = 1.f, bwd = 1.f;
    const bool conc = P.rate_form[r] == FDLBM_RATE_CONC_BILINEAR;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const float v = conc ? Cw[j] : Cw[j] * iCt;
      const int nu = P.nu[r][j];
      for (int q = 0; q < -nu; ++q) fwd *= v;
      for (int q = 0; q < nu; ++q) bwd *= v;
    }
    rate[r] = conc ? kr[r] * fwd : kr[r] * (fwd - bwd * P.inv_Keq[r]);
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

// One solid node (compact index n, entry idx of the solid list): FD heat step;
// interface wall nodes also run the reactive diffusive wall. Ledger increments accumulate
// into acc (Q_rxn, Q_wall, Q_couple, Q_fixedT, non-converged iterations). rw_prev
// [ns][n_wall_list] holds each catalytic wall's converged density of the previous step
// (NaN before the first step), the start of its iteration.
// A moving wall (wall_u != nullptr: velocity per wall-list entry) emits f^eq_j(1, U_w, T_w)
// of each species instead of the rest weights (Eq. BC_g_ji_1 with the wall velocity).
__device__ __forceinline__ float wmove(int i, float sM, float M, float2 u, float T) {
  const float fx = EX(i) == 0 ? 1.f - M * u.x * u.x - T : 0.5f * (float(EX(i)) * sM * u.x + M * u.x * u.x + T);
  const float fy = EY(i) == 0 ? 1.f - M * u.y * u.y - T : 0.5f * (float(EY(i)) * sM * u.y + M * u.y * u.y + T);
  return fx * fy;
}

// Deviations of the emitted shapes from the rest weights W0_i at T_ref, formed from the
// wall temperature's deviation d = T_w - T_ref: with 1D factors f = f0 + df, the product
// f_x f_y - f0_x f0_y = f0_x df_y + df_x f0_y + df_x df_y.
__device__ __forceinline__ float dwrest(const DevParams& P, int i, float d) {
  const float fx0 = EX(i) == 0 ? 1.f - P.Tref : 0.5f * P.Tref, fy0 = EY(i) == 0 ? 1.f - P.Tref : 0.5f * P.Tref;
  const float dfx = EX(i) == 0 ? -d : 0.5f * d, dfy = EY(i) == 0 ? -d : 0.5f * d;
  return fmaf(fx0, dfy, dfx * (fy0 + dfy));
}
__device__ __forceinline__ float dwmove(const DevParams& P, int i, float sM, float M, float2 u, float d) {
  const float fx0 = EX(i) == 0 ? 1.f - P.Tref : 0.5f * P.Tref, fy0 = EY(i) == 0 ? 1.f - P.Tref : 0.5f * P.Tref;
  const float mx = M * u.x * u.x, my = M * u.y * u.y;
  const float dfx = EX(i) == 0 ? -(mx + d) : 0.5f * (float(EX(i)) * sM * u.x + mx + d);
  const float dfy = EY(i) == 0 ? -(my + d) : 0.5f * (float(EY(i)) * sM * u.y + my + d);
  return fmaf(fx0, dfy, dfx * (fy0 + dfy));
}

template <class PT, int NS, bool DET = false>
__device__ __forceinline__ void solid_node(const DevParams& P, const PT* __restrict__ src, PT* __restrict__ dst,
                                           const float* __restrict__ Ts_src, float* __restrict__ Ts_dst,
                                           const uint32_t* __restrict__ code, const float* __restrict__ Tgas, int n,
                                           double (&acc)[LG_COUNT], float* __restrict__ rw_prev, int idx,
                                           uint32_t step, const float2* __restrict__ wall_u) {
  {
    const int x = n % P.nx, y = n / P.nx;
    const int k = pad_index(P, x, y);
    const uint32_t cw = __ldg(code + k);
    const float Tx = Ts_src[n];
    float lap = 0.f, gas_term = 0.f;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int ox = d == 0 ? 1 : d == 1 ? -1 : 0;
      const int oy = d == 2 ? 1 : d == 3 ? -1 : 0;
      // neighbour class bits of solid nodes: bit NBR_GAS_SHIFT + (i - 1) set for a solid
      // neighbour along direction i = 1..4 (+x, +y, -x, -y)
      const int i = d == 0 ? 1 : d == 1 ? 3 : d == 2 ? 2 : 4;
      if ((cw >> (NBR_GAS_SHIFT + i - 1)) & 1u) {
        lap += Ts_src[lat_index(P, x + ox, y + oy)] - Tx;
        continue;
      }
      const int nb = lat_index(P, x + ox, y + oy);
      if (nb < 0) {
        const int face = d == 0 ? 1 : d == 1 ? 0 : d == 2 ? 3 : 2;
        if (P.fixedT_face[face]) {
          lap += P.dTout - Tx;
          acc[LG_QFIXEDT] += double(P.rhocp_s) * double(P.alpha_s) * double(P.dTout - Tx);
        }
        continue;
      }
      if (Tgas != nullptr && node_class(__ldg(code + k + ox + oy * P.pitch)) == GAS)
        gas_term += Tgas[nb] - Tx;
    }
    float Tn = fmaf(P.alpha_s, lap, Tx);
    if (node_class(cw) == WALL) {
      const float Tw = P.Tref + Tx;
      // Arrival directions carry a stencil code; the wall emits along the opposite
      // directions (towards its gas neighbours).
      uint32_t arr = 0;
      for (int i = 1; i < Q; ++i)
        if (stencil_of(cw, i) != ST_NOT_ARRIVAL) arr |= 1u << i;
      // Emitted shape at the wall temperature, W0_i + dW_i, with dW_i formed from the
      // deviation Tx so that FP32 keeps its digits; B = sum of the shape, dB of dW.
      float B = 0.f, dB = 0.f;
      for (int i = 1; i < Q; ++i)
        if (arr & (1u << OPP(i))) {
          B += wrest(i, Tw);
          dB += dwrest(P, i, Tx);
        }
      float A[NS], Ah[NS], rw[NS], mj[NS];
      float Earr = 0.f, W0arr = 0.f;
#pragma unroll
      for (int j = 0; j < NS; ++j) Ah[j] = 0.f;
      // Populations arriving from the gas: all lanes of a warp step through the directions
      // together, so that their loads of one direction plane coalesce; branch-free
      // stencils, loads of all species issued together.
#pragma unroll 1
      for (int i = 1; i < Q; ++i) {
        if (!(arr & (1u << i))) continue;
        const int off = EX(i) + EY(i) * P.pitch;
        const StencilCoef sc = stencil_coef(stencil_of(cw, i));
        const int dA = sc.mA * off, dB = sc.mB * off;
        const float e2h = 0.5f * float(EX(i) * EX(i) + EY(i) * EY(i));
        W0arr += P.W0[i];
        float v1[NS], vA[NS], vB[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          const int b = (j * Q + i) * (int)P.plane + k;
          v1[j] = pop_ld(src + (b - off), P.hsi[j]);
          vA[j] = pop_ld(src + (b + dA), P.hsi[j]);
          vB[j] = pop_ld(src + (b + dB), P.hsi[j]);
        }
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          float v = v1[j];
          if (!P.onlattice[j]) {
            const float d1 = fmaf(-sc.p1, v1[j], fmaf(sc.pA, vA[j], sc.pB * vB[j]));
            const float d2 = fmaf(-sc.q1, v1[j], fmaf(sc.qA, vA[j], sc.qB * vB[j]));
            v = fmaf(P.ha[j], d1, fmaf(P.ha2[j], d2, v1[j]));
          }
          if constexpr (DET) {  // arrival's departure from the shift; its energy, exactly
            const double e = eps_weight(P, j, EX(i) * EX(i) + EY(i) * EY(i));
            acc[LG_DINT] += e * (double(v) - double(v1[j]));
            acc[LG_QWALLX] -= e * (double(v) + double(P.rref[j]) * double(P.W0[i]));
          }
          Ah[j] += v;  // deviations; the rest part rref W0 is added below
          Earr = fmaf(e2h * P.c2[j], v, Earr);
        }
      }
      // normalisation of the emitted shape: 1 / B, per species for a moving wall
      float iBj[NS], dBj[NS];
      const bool moving = wall_u != nullptr;
      float2 uw = make_float2(0.f, 0.f);
      if (moving) {
        uw = wall_u[idx];
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          float Bj = 0.f, dbj = 0.f;
          for (int i = 1; i < Q; ++i)
            if (arr & (1u << OPP(i))) {
              Bj += wmove(i, P.sqrtM[j], P.M[j], uw, Tw);
              dbj += dwmove(P, i, P.sqrtM[j], P.M[j], uw, Tx);
            }
          iBj[j] = 1.f / Bj;
          dBj[j] = dbj;
        }
      } else {
        const float iB = 1.f / B;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          iBj[j] = iB;
          dBj[j] = dB;
        }
      }
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        A[j] = fmaf(P.rref[j], W0arr, Ah[j]);
        rw[j] = A[j] * iBj[j];
        mj[j] = 0.f;
      }
      float rate[MAX_NR] = {0.f, 0.f, 0.f, 0.f};
      const bool cat = (cw & CATALYTIC_BIT) && P.nr > 0;
      if (cat) {
        float kr[MAX_NR];
        const float TK = P.T3T0 * Tw;
        for (int r = 0; r < P.nr; ++r) kr[r] = P.k0[r] * expf(-P.EaR[r] / TK);
        // Start from the previous step's converged density when there is one (the fixed
        // point moves little between steps); the converged value does not depend on the
        // start.
        float* rp = rw_prev + idx;
        if (rp[0] == rp[0]) {
#pragma unroll
          for (int j = 0; j < NS; ++j) rw[j] = rp[(long long)j * P.n_wall_list];
        }
        bool conv = false;
        for (int it = 0; it < P.rho_w_maxit; ++it) {
          rates<NS>(P, rw, kr, rate);
          float d = 0.f, rmax = 0.f;
#pragma unroll
          for (int j = 0; j < NS; ++j) {
            float mm = 0.f;
            for (int r = 0; r < P.nr; ++r) mm += P.M[j] * float(P.nu[r][j]) * rate[r];
            const float nw = (A[j] + mm) * iBj[j];
            d = fmaxf(d, fabsf(nw - rw[j]));
            rmax = fmaxf(rmax, fabsf(nw));
            rw[j] = nw;
          }
          if (d <= fmaxf(P.rho_w_tol, 4.f * FLT_EPSILON * rmax)) { conv = true; break; }
        }
        if (!conv) acc[LG_NOCONV] += 1.0;
#pragma unroll
        for (int j = 0; j < NS; ++j) rp[(long long)j * P.n_wall_list] = rw[j];
        rates<NS>(P, rw, kr, rate);
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          float mm = 0.f;
          for (int r = 0; r < P.nr; ++r) mm += P.M[j] * float(P.nu[r][j]) * rate[r];
          mj[j] = mm;
        }
      }
      const Ghost gh = ghost_of(P, x, y);
      const uint32_t seed = sizeof(PT) == 4 ? 0U : node_seed(k, step);
      float Eout = 0.f;
      // emitted deviation dscale W0_i + (rref + dscale) dW_i with dscale = (A + m) / B -
      // rref = (sum of arrived deviations - rref dB + m) / B: the rest parts rref W0 of
      // the arrivals and of the emissions cancel (the two direction sets mirror each
      // other), so only small quantities are rounded.
      float dsc[NS];
#pragma unroll
      for (int j = 0; j < NS; ++j) dsc[j] = (fmaf(-P.rref[j], dBj[j], Ah[j]) + mj[j]) * iBj[j];
      // Emissions towards the gas neighbours (the directions opposite to the arrivals).
#pragma unroll 1
      for (int i = 1; i < Q; ++i) {
        if (!(arr & (1u << OPP(i)))) continue;
        const float dwr = dwrest(P, i, Tx);
        const float e2h = 0.5f * float(EX(i) * EX(i) + EY(i) * EY(i));
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          const float dw = moving ? dwmove(P, i, P.sqrtM[j], P.M[j], uw, Tx) : dwr;
          const float dv = fmaf(dsc[j], P.W0[i], (P.rref[j] + dsc[j]) * dw);
          pop_store_ghosts(dst + (long long)(j * Q + i) * P.plane, k, gh, dv, P.hs[j], seed, j * Q + i);
          if constexpr (DET)  // FP32 storage: dv is the value stored
            acc[LG_QWALLX] += eps_weight(P, j, EX(i) * EX(i) + EY(i) * EY(i)) *
                              (double(dv) + double(P.rref[j]) * double(P.W0[i]));
          Eout = fmaf(e2h * P.c2[j], dv, Eout);
        }
      }
      float q = 0.f;
      if (cat)
        for (int r = 0; r < P.nr; ++r) q += P.heat[r] * rate[r];
      const float dE = Eout - Earr;  // energy the wall put into the gas (deviation sums)
      const float couple = P.coupling == FDLBM_COUPLING_PAPER ? P.kappa_f * gas_term : -dE;
      Tn += (q + couple) * P.inv_rhocp_s;
      acc[LG_QRXN] += q;
      acc[LG_QWALL] += dE;
      acc[LG_QCOUPLE] += couple;
    }
    Ts_dst[n] = Tn;
    if constexpr (DET) acc[LG_DH] += double(P.rhocp_s) * (double(Tn) - double(Tx));
  }
}

// Block-level sum of the first NQ ledger increments into this block's own slot (no
// atomics; the slots are summed when the ledger is read). The plain step keeps the first
// LG_BASIC; the exact-accounts step all LG_COUNT.
constexpr int LG_BASIC = LG_NOCONV + 1;
template <int NQ = LG_BASIC>
__device__ __forceinline__ void ledger_block_store(double (&acc)[LG_COUNT], double* __restrict__ slot) {
  __shared__ double sh[NQ][GB / 32];
  // FP64 arithmetic is slow on this part: quantities that are zero in the whole warp
  // (interior solid nodes away from fixed-T faces contribute nothing) skip the shuffles.
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    if (__any_sync(0xffffffffu, acc[q] != 0.0))
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[q][warp] = acc[q];
  __syncthreads();
  if (threadIdx.x < NQ) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
    if (v != 0.0) slot[threadIdx.x] += v;
  }
}

// One time step in one launch. Every block takes a role from its descriptor: gas blocks
// run a gas tile (its interior and halo entries of the gas list), solid blocks {1, first
// list entry, count} the wall + FD update of consecutive solid nodes. The host
// interleaves the descriptors by row bands so that wall blocks follow the gas tiles of
// the same rows and find their neighbours' populations in L2. MODE 1: only the gas tiles
// run, recomputing the pre-collision moments into mom.
template <class PT, int NS, bool PHI, bool LT = false, bool DET = false, int MODE = 0>
__global__ void __launch_bounds__(GB, GAS_MIN_BLOCKS) step_kernel(
    DevParams P, const PT* __restrict__ src, PT* __restrict__ dst, const uint32_t* __restrict__ code,
    const int2* __restrict__ gas_list, const uint16_t* __restrict__ gas_slot, const int32_t* __restrict__ solid_list,
    const int4* __restrict__ blocks, float* __restrict__ mom, const float* __restrict__ Ts_src,
    float* __restrict__ Ts_dst, const float* __restrict__ Tgas_src, float* __restrict__ Tgas_dst,
    double* __restrict__ ledger, int* __restrict__ flags, float* __restrict__ rw_prev, uint32_t step,
    const float2* __restrict__ wall_u) {
  extern __shared__ float smem[];
  const int4 d = __ldg(blocks + blockIdx.x);
  const int tid = threadIdx.x;
  if (d.x == 0) {
    if constexpr (DET && MODE == 0) {
      Acct ac{0.0, 0.0, 0.0, 0.0};
      gas_tile<PT, NS, PHI, 0, LT, true>(P, src, dst, code, gas_list, gas_slot, d, nullptr, Tgas_dst, flags, smem,
                                         step, &ac);
      double acc[LG_COUNT];
#pragma unroll
      for (int q = 0; q < LG_COUNT; ++q) acc[q] = 0.0;
      acc[LG_QIN] = ac.qin;
      acc[LG_QOUT] = ac.qout;
      acc[LG_DINT] = ac.dint;
      acc[LG_DCOL] = ac.dcol;
      ledger_block_store<LG_COUNT>(acc, ledger + (long long)blockIdx.x * LG_COUNT);
    } else {
      gas_tile<PT, NS, PHI, MODE, LT>(P, src, dst, code, gas_list, gas_slot, d, mom, Tgas_dst, flags, smem, step);
    }
    return;
  }
  if constexpr (MODE == 0) {
    double acc[LG_COUNT];
#pragma unroll
    for (int q = 0; q < LG_COUNT; ++q) acc[q] = 0.0;
    if (tid < d.z)
      solid_node<PT, NS, DET>(P, src, dst, Ts_src, Ts_dst, code, Tgas_src, __ldg(solid_list + d.y + tid), acc, rw_prev,
                              d.y + tid, step, wall_u);
    ledger_block_store<DET ? LG_COUNT : LG_BASIC>(acc, ledger + (long long)blockIdx.x * LG_COUNT);
  }
}

// Batched time step: several independent lattices (members of a batch) advance in one
// launch. A descriptor {2 member + role, first, count, member-local block index} selects
// the member; the block copies the member's parameters into shared memory and takes its
// buffers from the member's device state. members[m] = {buffer holding time level t when
// counter = 0, step index when counter = 0}; counter counts the batch's steps (advanced
// by batch_advance after every step), so one captured launch sequence serves every step.
template <class PT, int NS, bool PHI>
__global__ void __launch_bounds__(GB, GAS_MIN_BLOCKS) step_kernel_batch(
    const DevParams* __restrict__ params, const DevState* __restrict__ states, const int2* __restrict__ members,
    const int4* __restrict__ blocks, const uint32_t* __restrict__ counter) {
  extern __shared__ float smem[];
  __shared__ DevParams sP;
  const int4 d = __ldg(blocks + blockIdx.x);
  const int m = d.x >> 1;
  {
    const int* from = reinterpret_cast<const int*>(params + m);
    int* to = reinterpret_cast<int*>(&sP);
    for (int w = threadIdx.x; w < int(sizeof(DevParams) / sizeof(int)); w += blockDim.x) to[w] = __ldg(from + w);
  }
  __syncthreads();
  const DevParams& P = sP;
  const DevState& S = states[m];
  const uint32_t c = *counter;
  const int2 mm = __ldg(members + m);
  const int src = (mm.x + int(c & 1U)) & 1, dstb = src ^ 1;
  const uint32_t step = uint32_t(mm.y) + c;
  const PT* hs = static_cast<const PT*>(S.h[src]);
  PT* hd = static_cast<PT*>(S.h[dstb]);
  const bool paper = P.coupling == FDLBM_COUPLING_PAPER;
  const int tid = threadIdx.x;
  if ((d.x & 1) == 0) {
    gas_tile<PT, NS, PHI, 0>(P, hs, hd, S.code, S.gas_list, S.gas_slot, d, nullptr,
                             paper ? S.Tgas + (long long)dstb * P.n : nullptr, S.flags, smem, step);
    return;
  }
  double acc[LG_COUNT];
#pragma unroll
  for (int q = 0; q < LG_COUNT; ++q) acc[q] = 0.0;
  if (tid < d.z)
    solid_node<PT, NS>(P, hs, hd, S.Ts[src], S.Ts[dstb], S.code, paper ? S.Tgas + (long long)src * P.n : nullptr,
                       __ldg(S.solid_list + d.y + tid), acc, S.rw, d.y + tid, step, S.wall_u);
  ledger_block_store(acc, S.ledger + (long long)d.w * LG_COUNT);
}

__global__ void batch_advance(uint32_t* counter) { *counter += 1U; }

// ---------------------------------------------------------------------------------------
// Initialisation (FP64 arithmetic, then rounded), over every padded cell so that ghost
// copies start consistent.
// ---------------------------------------------------------------------------------------
__device__ double wfac_d(int e, double v, double M, double T) {
  return e == 0 ? 1.0 - M * v * v - T : 0.5 * (double(e) * sqrt(M) * v + M * v * v + T);
}

template <class PT>
__global__ void init_kernel(DevParams P, PT* __restrict__ h0, PT* __restrict__ h1,
                            float* __restrict__ Ts0, float* __restrict__ Ts1, float* __restrict__ mom,
                            float* __restrict__ Tgas, const uint32_t* __restrict__ code,
                            const double* __restrict__ X, const double* __restrict__ u,
                            const double* __restrict__ Tl, const double* __restrict__ Tsl,
                            const double* __restrict__ Cn, const double* __restrict__ inlet_u,
                            const double* __restrict__ X_inlet, double Tref) {
  const long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (kk >= P.plane) return;
  const int k = int(kk);
  for (int j = 0; j < P.ns; ++j)
    for (int i = 0; i < Q; ++i) {
      h0[(long long)(j * Q + i) * P.plane + k] = pop_enc<PT>(0.f, 1.f);
      h1[(long long)(j * Q + i) * P.plane + k] = pop_enc<PT>(0.f, 1.f);
    }
  if (k >= P.pitch * (P.ny + 2 * P.yoff)) return;
  const int px = k % P.pitch, py = k / P.pitch;
  int x = px - P.xoff, y = py - P.yoff;
  // Ghost cells within GHOST of a periodic face take the wrapped node's state.
  if (x < 0 || x >= P.nx) {
    if (!P.periodic_x || x < -GHOST || x >= P.nx + GHOST) return;
    x = x < 0 ? x + P.nx : x - P.nx;
  }
  if (y < 0 || y >= P.ny) {
    if (!P.periodic_y || y < -GHOST || y >= P.ny + GHOST) return;
    y = y < 0 ? y + P.ny : y - P.ny;
  }
  const bool real = px - P.xoff == x && py - P.yoff == y;
  const int n = x + P.nx * y;
  const uint32_t cw = code[pad_index(P, x, y)];
  const uint32_t c = node_class(cw);
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
  if (c == GAS || c == INLET || c == OUTLET) {
    for (int j = 0; j < P.ns; ++j) {
      const double M = P.M[j];
      const double rho = C * Xn[j] * M;
      for (int i = 0; i < Q; ++i) {
        const double f = rho * wfac_d(EX(i), ux, M, T) * wfac_d(EY(i), uy, M, T);
        const double w0 = (EX(i) == 0 ? 1.0 - Tref : 0.5 * Tref) * (EY(i) == 0 ? 1.0 - Tref : 0.5 * Tref);
        const PT v = pop_enc<PT>(float(f - double(P.rref[j]) * w0), P.hs[j]);
        h0[(long long)(j * Q + i) * P.plane + k] = v;
        h1[(long long)(j * Q + i) * P.plane + k] = v;
      }
    }
    if (c == GAS && real) {
      for (int j = 0; j < P.ns; ++j) mom[(long long)j * P.n + n] = float(C * Xn[j] * P.M[j]);
      mom[(long long)P.ns * P.n + n] = float(ux);
      mom[(long long)(P.ns + 1) * P.n + n] = float(uy);
      mom[(long long)(P.ns + 2) * P.n + n] = float(T - Tref);
      Tgas[n] = Tgas[P.n + n] = float(T - Tref);
    }
  } else if (c == WALL || c == SOLID) {
    const double Ts = Tsl[n];
    if (real) Ts0[n] = Ts1[n] = float(Ts - Tref);
    if (c == WALL) {
      for (int j = 0; j < P.ns; ++j) {
        const double rho = C * Xn[j] * P.M[j];
        for (int i = 1; i < Q; ++i) {
          if (stencil_of(cw, OPP(i)) == ST_NOT_ARRIVAL) continue;
          const double wr = (EX(i) == 0 ? 1.0 - Ts : 0.5 * Ts) * (EY(i) == 0 ? 1.0 - Ts : 0.5 * Ts);
          const double w0 = (EX(i) == 0 ? 1.0 - Tref : 0.5 * Tref) * (EY(i) == 0 ? 1.0 - Tref : 0.5 * Tref);
          const PT v = pop_enc<PT>(float(rho * wr - double(P.rref[j]) * w0), P.hs[j]);
          h0[(long long)(j * Q + i) * P.plane + k] = v;
          h1[(long long)(j * Q + i) * P.plane + k] = v;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Outputs and reductions (compact node indices)
// ---------------------------------------------------------------------------------------
template <class PT>
__global__ void populations_out_kernel(DevParams P, const PT* __restrict__ h, float* __restrict__ dst) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)P.ns * Q * P.n;
  if (q >= total) return;
  const int n = int(q % P.n);
  const int ji = int(q / P.n);
  const int j = ji / Q, i = ji % Q;
  dst[q] = pop_ld(h + ((long long)ji * P.plane + pad_index(P, n % P.nx, n / P.nx)), P.hsi[j]) + P.rref[j] * P.W0[i];
}

// Ledger totals: E_gas (f-moments + in-transit wall emissions), H_solid, mass_j, moles_j.
template <class PT>
__global__ void totals_kernel(DevParams P, const float* __restrict__ mom, const PT* __restrict__ h,
                              const float* __restrict__ Ts, const uint32_t* __restrict__ code,
                              double* __restrict__ out) {
  __shared__ double sh[8];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int ns = P.ns;
  const long long N = P.n;
  double E = 0.0, H = 0.0, mass[MAX_NS], moles[MAX_NS];
  for (int j = 0; j < ns; ++j) mass[j] = moles[j] = 0.0;
  if (n < P.n) {
    const int k = pad_index(P, n % P.nx, n / P.nx);
    const uint32_t cw = code[k];
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
      const double ux = mom[ns * N + n], uy = mom[(ns + 1) * N + n], T = double(P.Tref) + mom[(ns + 2) * N + n];
      E = C * T + 0.5 * r * (ux * ux + uy * uy);
    } else if (c == WALL || c == SOLID) {
      H = double(P.rhocp_s) * (double(P.Tref) + double(Ts[n]));
      if (c == WALL) {
        for (int i = 1; i < Q; ++i) {
          if (stencil_of(cw, OPP(i)) == ST_NOT_ARRIVAL) continue;
          for (int j = 0; j < ns; ++j) {
            const double w = double(pop_ld(h + ((long long)(j * Q + i) * P.plane + k), P.hsi[j])) + double(P.rref[j]) * double(P.W0[i]);
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

template <class PT, int NS, bool PHI, bool LT = false, bool DET = false, int MODE = 0>
cudaError_t step_launch(const DevParams& P, const DevState& S, int src, cudaStream_t st, uint32_t step) {
  if (P.n_blocks <= 0) return cudaSuccess;
  const size_t smem = gas_smem_bytes<NS, LT>();
  static unsigned long long configured = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && !(configured & (1ull << dev))) {
    e = cudaFuncSetAttribute(step_kernel<PT, NS, PHI, LT, DET, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    configured |= 1ull << dev;
  }
  const int dstb = 1 - src;
  const bool paper = MODE == 0 && P.coupling == FDLBM_COUPLING_PAPER;
  step_kernel<PT, NS, PHI, LT, DET, MODE><<<P.n_blocks, P.block_threads, smem, st>>>(
      P, (const PT*)S.h[src], (PT*)S.h[dstb], S.code, S.gas_list, S.gas_slot, S.solid_list, S.blocks,
      MODE == 1 ? S.mom : nullptr, S.Ts[src], S.Ts[dstb], paper ? S.Tgas + (long long)src * P.n : nullptr,
      paper ? S.Tgas + (long long)dstb * P.n : nullptr, S.ledger, S.flags, S.rw, step, S.wall_u);
  return cudaGetLastError();
}

// Locally updated relaxation times and the exact-accounts step run the FP32 kernels
// instantiated in fdlbm_local_tau.cu and fdlbm_ledger_detail.cu (the host rejects other
// storage types).
// MODE 1 is the moments-only pass (the pre-collision moments of the step that reads src).
template <class PT, int NS, int MODE>
cudaError_t step_ns(const DevParams& P, const DevState& S, int src, cudaStream_t st, uint32_t step) {
  const bool phi = P.energy_correction != 0;
  if constexpr (sizeof(PT) == 4) {
    if (MODE == 0 && P.ledger_detail) return launch_step_detail(P, S, src, st, step);
    if (P.local_tau) return launch_step_local_tau(P, S, src, MODE == 1, st, step);
  }
  return phi ? step_launch<PT, NS, true, false, false, MODE>(P, S, src, st, step)
             : step_launch<PT, NS, false, false, false, MODE>(P, S, src, st, step);
}

template <class PT, int MODE>
cudaError_t dispatch_step(const DevParams& P, const DevState& S, int src, cudaStream_t st, uint32_t step) {
  switch (P.ns) {
    case 1: return step_ns<PT, 1, MODE>(P, S, src, st, step);
    case 2: return step_ns<PT, 2, MODE>(P, S, src, st, step);
    case 3: return step_ns<PT, 3, MODE>(P, S, src, st, step);
    case 4: return step_ns<PT, 4, MODE>(P, S, src, st, step);
    case 5: return step_ns<PT, 5, MODE>(P, S, src, st, step);
    case 6: return step_ns<PT, 6, MODE>(P, S, src, st, step);
    default: return cudaErrorInvalidValue;
  }
}


// ---------------------------------------------------------------------------------------
// Allocation-free totals. The per-node sums are those of totals_kernel; each block
// writes its partial sums to its own row of a fixed static scratch array (no atomics,
// nothing to clear beforehand), and one block then adds the rows in block order, so the
// result does not depend on the order in which blocks ran.

// Partial sums of block b: E_gas, H_solid, mass[ns], moles[ns] at row b.
template <class PT>
__global__ void __launch_bounds__(TOTALS_STATIC_BLOCK)
totals_partial_kernel(DevParams P, const float* __restrict__ mom, const PT* __restrict__ h,
                      const float* __restrict__ Ts, const uint32_t* __restrict__ code,
                      double* __restrict__ part) {
  __shared__ double sh[TOTALS_STATIC_BLOCK / 32];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int ns = P.ns, cnt = 2 + 2 * ns;  // E_gas, H_solid, mass[ns], moles[ns]
  const long long N = P.n;
  double E = 0.0, H = 0.0, mass[MAX_NS], moles[MAX_NS];
  for (int j = 0; j < ns; ++j) mass[j] = moles[j] = 0.0;
  if (n < P.n) {
    const int k = pad_index(P, n % P.nx, n / P.nx);
    const uint32_t cw = code[k];
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
      const double ux = mom[ns * N + n], uy = mom[(ns + 1) * N + n], T = double(P.Tref) + mom[(ns + 2) * N + n];
      E = C * T + 0.5 * r * (ux * ux + uy * uy);
    } else if (c == WALL || c == SOLID) {
      H = double(P.rhocp_s) * (double(P.Tref) + double(Ts[n]));
      if (c == WALL) {
        // populations emitted by the wall and not yet streamed into the gas
        for (int i = 1; i < Q; ++i) {
          if (stencil_of(cw, OPP(i)) == ST_NOT_ARRIVAL) continue;
          for (int j = 0; j < ns; ++j) {
            const double w = double(pop_ld(h + ((long long)(j * Q + i) * P.plane + k), P.hsi[j])) + double(P.rref[j]) * double(P.W0[i]);
            mass[j] += w;
            moles[j] += w / double(P.M[j]);
            E += 0.5 * double(P.c2[j]) * double(EX(i) * EX(i) + EY(i) * EY(i)) * w;
          }
        }
      }
    }
  }
  double* row = part + (long long)blockIdx.x * cnt;
  double s = block_sum(E, sh);
  if (threadIdx.x == 0) row[0] = s;
  s = block_sum(H, sh);
  if (threadIdx.x == 0) row[1] = s;
  for (int j = 0; j < ns; ++j) {
    s = block_sum(mass[j], sh);
    if (threadIdx.x == 0) row[2 + j] = s;
    s = block_sum(moles[j], sh);
    if (threadIdx.x == 0) row[2 + ns + j] = s;
  }
}

template <class PT, int NS, bool PHI>
cudaError_t batch_launch(const BatchLaunch& B, cudaStream_t st) {
  if (B.n_blocks <= 0) return cudaSuccess;
  const size_t smem = gas_smem_bytes<NS>();
  static unsigned long long configured = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && !(configured & (1ull << dev))) {
    e = cudaFuncSetAttribute(step_kernel_batch<PT, NS, PHI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured |= 1ull << dev;
  }
  step_kernel_batch<PT, NS, PHI><<<B.n_blocks, GB, smem, st>>>(B.params, B.states, B.members, B.blocks, B.counter);
  batch_advance<<<1, 1, 0, st>>>(B.counter);
  return cudaGetLastError();
}

template <class PT>
cudaError_t dispatch_batch(const BatchLaunch& B, cudaStream_t st) {
  const bool phi = B.energy_correction != 0;
  switch (B.ns) {
    case 1: return phi ? batch_launch<PT, 1, true>(B, st) : batch_launch<PT, 1, false>(B, st);
    case 2: return phi ? batch_launch<PT, 2, true>(B, st) : batch_launch<PT, 2, false>(B, st);
    case 3: return phi ? batch_launch<PT, 3, true>(B, st) : batch_launch<PT, 3, false>(B, st);
    case 4: return phi ? batch_launch<PT, 4, true>(B, st) : batch_launch<PT, 4, false>(B, st);
    case 5: return phi ? batch_launch<PT, 5, true>(B, st) : batch_launch<PT, 5, false>(B, st);
    case 6: return phi ? batch_launch<PT, 6, true>(B, st) : batch_launch<PT, 6, false>(B, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Entry points of one storage type (explicitly instantiated once per type).
template <class PT>
cudaError_t storage_init(const DevParams& P, const DevState& S, const double* X, const double* u,
                         const double* T_lat, const double* Ts_lat, const double* C, const double* inlet,
                         cudaStream_t st) {
  const double* X_inlet = inlet + P.ny;
  const long long nb = (P.plane + 255) / 256;
  init_kernel<PT><<<(unsigned)nb, 256, 0, st>>>(P, (PT*)S.h[0], (PT*)S.h[1], S.Ts[0], S.Ts[1], S.mom,
                                               S.Tgas, S.code, X, u, T_lat, Ts_lat, C, inlet, X_inlet,
                                               double(P.Tref));
  return cudaGetLastError();
}

template <class PT>
cudaError_t storage_step(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st,
                         uint32_t step) {
  if (moments_only) return dispatch_step<PT, 1>(P, S, src, st, step);
  return dispatch_step<PT, 0>(P, S, src, st, step);
}

template <class PT>
cudaError_t storage_batch_step(const BatchLaunch& B, cudaStream_t st) {
  return dispatch_batch<PT>(B, st);
}

template <class PT>
cudaError_t storage_populations_out(const DevParams& P, const DevState& S, int cur, float* dst, cudaStream_t st) {
  const long long total = (long long)P.ns * Q * P.n;
  const int nb = int((total + 255) / 256);
  populations_out_kernel<PT><<<nb, 256, 0, st>>>(P, (const PT*)S.h[cur], dst);
  return cudaGetLastError();
}

template <class PT>
cudaError_t storage_totals(const DevParams& P, const DevState& S, int cur, cudaStream_t st) {
  const int nb = (P.n + 255) / 256;
  totals_kernel<PT><<<nb, 256, 0, st>>>(P, S.mom, (const PT*)S.h[cur], S.Ts[cur], S.code, S.red);
  return cudaGetLastError();
}

template <class PT>
cudaError_t storage_totals_partial(const DevParams& P, const DevState& S, int cur, double* part, int nb,
                                   cudaStream_t st) {
  totals_partial_kernel<PT><<<nb, TOTALS_STATIC_BLOCK, 0, st>>>(P, S.mom, (const PT*)S.h[cur], S.Ts[cur], S.code, part);
  return cudaGetLastError();
}

#define FDLBM_STORAGE_ENTRY_POINTS(PREFIX, PT)                                                                    \
  PREFIX template cudaError_t storage_init<PT>(const DevParams&, const DevState&, const double*, const double*,  \
                                              const double*, const double*, const double*, const double*,        \
                                              cudaStream_t);                                                     \
  PREFIX template cudaError_t storage_step<PT>(const DevParams&, const DevState&, int, bool, cudaStream_t,       \
                                              uint32_t);                                                         \
  PREFIX template cudaError_t storage_batch_step<PT>(const BatchLaunch&, cudaStream_t);                          \
  PREFIX template cudaError_t storage_populations_out<PT>(const DevParams&, const DevState&, int, float*,         \
                                                         cudaStream_t);                                          \
  PREFIX template cudaError_t storage_totals<PT>(const DevParams&, const DevState&, int, cudaStream_t);           \
  PREFIX template cudaError_t storage_totals_partial<PT>(const DevParams&, const DevState&, int, double*, int,    \
                                                        cudaStream_t);

}  // namespace fdlbm
