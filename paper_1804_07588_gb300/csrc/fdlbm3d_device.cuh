// Device code of the coupled FD-LBM solver on the D3Q19 lattice (sm_103a), templated on
// the population storage type PT (float, __nv_bfloat16, __half). Included by
// fdlbm3d_kernels.cu (FP32 and the launchers) and fdlbm3d_store_{bf16,fp16}.cu.
//
// The paper states its scheme on D2Q9 and announces the 3D extension (Sec. 2). The
// 3D lattice takes the product-form equilibrium of Eq. eq_state_pop on D3Q27 and folds
// every corner population onto its three face diagonals (+), its three axis links (-)
// and the rest population (+), which keeps the moments up to second order. Summed by
// hand, with per-axis factors w(0) = 1 - M u^2 - T, w(+-1) = (+-sqrt(M) u + M u^2 + T)/2
// and S = w(+1) + w(-1) = M u^2 + T:
//   face diagonal (a on axis p, b on axis q):  rho w_p(a) w_q(b)
//   axis link (a on axis p; q, r the others):  rho w_p(a) (w_q(0) w_r(0) - S_q S_r)
//   rest:                                      rho (w_x(0) w_y(0) w_z(0) + S_x S_y S_z).
// The correction coefficients, the temperature and the energy-correction flux take
// D = 3: psi = +-1 on the axis links of its component and -sgn(c)/8 on the 8 face
// diagonals with that component (over c_j), phi = {-1 rest, 1/6 axis, 0 diagonal} / c_j^2,
// T_g = (E - J^2/rho) / (3 C), T = T_g + sum_j divq_j / (6 C), and
// K_j = (2 c_pj / Pr - 2 / M_j) tau1_j C_j T with c_pj = 5 / (2 M_j) (the folded product
// form carries 2/5 of the kinetic heat flux).
//
// Storage and kernels follow the D2Q9 path: populations as FP32 deviations from the
// rest equilibrium of the inlet state, SoA planes [species][direction] on a padded
// lattice with GHOST3 ghost layers (periodic copies written by the producing node), one
// fused step kernel per time step whose blocks take a gas role (one thread per entry of
// a compact gas-node list) or a solid role (interface wall nodes, then interior solid
// nodes), and an FP64 ledger with one slot row per block.
#pragma once

#include <cfloat>
#include <cmath>

// Population storage helpers (pop_ld, pop_round, pop_stcs, pop_enc, node_seed,
// pop_random) are shared with the D2Q9 kernels.
#include "fdlbm_device.cuh"

namespace fdlbm {

// The step that also keeps the exact accounts (FP32 storage; fdlbm3d_ledger_detail.cu), and
// the energy of the stored populations of gas nodes and wall emissions (into *out).
cudaError_t launch_step3_detail(const DevParams& P, const DevState& S, int src, cudaStream_t st, uint32_t step);
cudaError_t launch_pop_energy3(const DevParams& P, const DevState& S, int cur, double* out, cudaStream_t st);

namespace {

constexpr int G3 = STEP_BLOCK3;

// D3Q19 velocities: rest, axis links (+x -x +y -y +z -z), face diagonals; the opposite
// of i > 0 is i + 1 for odd i and i - 1 for even i.
__host__ __device__ constexpr int DX(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1 : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int DY(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1 : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int DZ(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1 : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int OPP3(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr int NNZ(int i) { return (DX(i) != 0) + (DY(i) != 0) + (DZ(i) != 0); }
__host__ __device__ constexpr int DC(int i, int a) { return a == 0 ? DX(i) : a == 1 ? DY(i) : DZ(i); }

__device__ __forceinline__ long long poff(const DevParams& P, int i) {
  return (long long)DX(i) + (long long)DY(i) * P.pitch + (long long)DZ(i) * P.slab;
}
__device__ __forceinline__ int pad3(const DevParams& P, int x, int y, int z) {
  return (x + P.xoff) + (y + P.yoff) * P.pitch + (int)((z + P.zoff) * P.slab);
}
__device__ __forceinline__ void xyz_of(const DevParams& P, int n, int& x, int& y, int& z) {
  x = n % P.nx;
  const int r = n / P.nx;
  y = r % P.ny;
  z = r / P.ny;
}
// Compact index of (x, y, z) wrapped on periodic axes; -1 off the lattice.
__device__ __forceinline__ int lat3(const DevParams& P, int x, int y, int z) {
  if (x < 0 || x >= P.nx) {
    if (!P.periodic_x) return -1;
    x = x < 0 ? x + P.nx : x - P.nx;
  }
  if (y < 0 || y >= P.ny) {
    if (!P.periodic_y) return -1;
    y = y < 0 ? y + P.ny : y - P.ny;
  }
  if (z < 0 || z >= P.nz) {
    if (!P.periodic_z) return -1;
    z = z < 0 ? z + P.nz : z - P.nz;
  }
  return x + P.nx * (y + P.ny * z);
}

// Padded-lattice shifts of the ghost copies a node at (x, y, z) writes: per axis the
// shift to the copy on the other side (0 when the node is not within GHOST3 of a
// periodic face); every combination of the non-zero shifts is a copy.
struct Ghost3 {
  int d[3];
};
__device__ __forceinline__ Ghost3 ghost3(const DevParams& P, int x, int y, int z) {
  Ghost3 g{{0, 0, 0}};
  if (P.periodic_x) g.d[0] = x < GHOST3 ? P.nx : (x >= P.nx - GHOST3 ? -P.nx : 0);
  if (P.periodic_y) g.d[1] = y < GHOST3 ? P.ny * P.pitch : (y >= P.ny - GHOST3 ? -P.ny * P.pitch : 0);
  if (P.periodic_z) g.d[2] = z < GHOST3 ? (int)(P.nz * P.slab) : (z >= P.nz - GHOST3 ? -(int)(P.nz * P.slab) : 0);
  return g;
}
// Streaming (evict-first) store of an encoded value e at k and at every ghost copy.
template <class T>
__device__ __forceinline__ void put3(T* p, int k, const Ghost3& g, bool ghosts, T e) {
  pop_stcs(p + k, e);
  if (!ghosts) return;
#pragma unroll
  for (int m = 1; m < 8; ++m) {
    const int sx = (m & 1) ? g.d[0] : 0, sy = (m & 2) ? g.d[1] : 0, sz = (m & 4) ? g.d[2] : 0;
    if (((m & 1) && !sx) || ((m & 2) && !sy) || ((m & 4) && !sz)) continue;
    pop_stcs(p + k + sx + sy + sz, e);
  }
}
__device__ __forceinline__ void store3(float* p, int k, const Ghost3& g, bool ghosts, float v) { put3(p, k, g, ghosts, v); }
// Store of a time-step result v of population q (stochastic rounding for 16-bit storage).
template <class PT>
__device__ __forceinline__ void pop_store3(PT* p, int k, const Ghost3& g, bool ghosts, float v, float sc,
                                           uint32_t seed, int q) {
  put3(p, k, g, ghosts, pop_round<PT>(v, sc, sizeof(PT) == 4 ? 0U : pop_random(seed, q)));
}

// Streaming stencils by code (central, forward, backward, linear-s0, linear-s2, none):
// pulled value s1 + (a/2) [pA sA + pB sB - p1 s1] + (a^2/2) [qA sA + qB sB - q1 s1],
// sA at x + mA e_i, sB at x + mB e_i (the branch-free form of Sec. 4.2's stencils).
__constant__ float4 c3_p[8] = {{0.f, 0.f, 0.f, 0.f},   {-1.f, 1.f, 0.f, 1.f}, {4.f, -1.f, 3.f, -2.f},
                               {-4.f, 1.f, -3.f, -2.f}, {2.f, 0.f, 2.f, 0.f},  {-2.f, 0.f, -2.f, 0.f},
                               {0.f, 0.f, 0.f, 0.f},    {0.f, 0.f, 0.f, 0.f}};
__constant__ float2 c3_q[8] = {{0.f, 0.f}, {1.f, 2.f}, {1.f, -1.f}, {1.f, -1.f},
                               {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f},  {0.f, 0.f}};
__constant__ int2 c3_m[8] = {{0, 0}, {-2, 0}, {0, 1}, {-2, -3}, {0, 0}, {-2, -2}, {0, 0}, {0, 0}};
// Direction table {ex, ey, ez, number of non-zero components}.
__constant__ int4 c3_e[Q19] = {{0, 0, 0, 0},  {1, 0, 0, 1},   {-1, 0, 0, 1},  {0, 1, 0, 1},   {0, -1, 0, 1},
                               {0, 0, 1, 1},  {0, 0, -1, 1},  {1, 1, 0, 2},   {-1, -1, 0, 2}, {1, -1, 0, 2},
                               {-1, 1, 0, 2}, {1, 0, 1, 2},   {-1, 0, -1, 2}, {1, 0, -1, 2},  {-1, 0, 1, 2},
                               {0, 1, 1, 2},  {0, -1, -1, 2}, {0, 1, -1, 2},  {0, -1, 1, 2}};

// Per-axis equilibrium factors and their deviations from the reference factors
// (W(0) = 1 - T_ref, W(+-1) = T_ref / 2, S_ref = T_ref).
struct Ax {
  float wp, wm, w0, S;       // w(+1), w(-1), w(0), S = w(+1) + w(-1)
  float dwp, dwm, dw0, dS;   // deviations from the reference factors
};
__device__ __forceinline__ Ax axis3(float sqrtM, float sMlo, float M, float v, float T, float dT) {
  const float s = fmaf(sqrtM, v, sMlo * v), m = M * v * v;
  Ax a;
  a.S = m + T;
  a.wp = 0.5f * (a.S + s);
  a.wm = 0.5f * (a.S - s);
  a.w0 = 1.f - a.S;
  a.dS = m + dT;
  a.dwp = 0.5f * (a.dS + s);
  a.dwm = 0.5f * (a.dS - s);
  a.dw0 = -a.dS;
  return a;
}

// Deviation of one species' folded equilibrium from rref W(T_ref), for all 19
// directions, density rho = rr + dr and per-axis factors A[3]:
//   face:  P_p(a) W(+-1) + (P_p(a) + rr W(+-1)) dw_q(b)
//   axis:  P_p(a) G0 + (P_p(a) + rr W(+-1)) dG_p,  G_p = w_q(0) w_r(0) - S_q S_r
//   rest:  dr R0 + (rr + dr) dR,  R = w_x(0) w_y(0) w_z(0) + S_x S_y S_z,
// with P_p(a) = rho w_p(a) - rr W(+-1) = dr W(+-1) + rho dw_p(a), G0 and R0 the rest values
// and the deviations dG, dR expanded so that no large term cancels. Density deviations
// multiply only rest factors: factors at the absolute temperature carry its rounding
// (~1.5e-8, nearly the same on all nodes of a uniform region), which multiplied by dr
// would act as a systematic energy source at every collision.
__device__ __forceinline__ void feq_dev3(float dr, float rr, float Tr, const Ax (&A)[3], float (&f)[Q19]) {
  const float W0 = 1.f - Tr, Wpm = 0.5f * Tr;
  // G0 = W0^2 - Tr^2 = 1 - 2 Tr and R0 = W0^3 + Tr^3 = 1 - 3 Tr W0, exact in FP32 for the
  // reference temperature on its 2^-12 grid
  const float rho = rr + dr, G0 = 1.f - 2.f * Tr, R0 = 1.f - 3.f * (Tr * W0);
  float Pp[3], Pm[3], dG[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    Pp[p] = fmaf(dr, Wpm, rho * A[p].dwp);
    Pm[p] = fmaf(dr, Wpm, rho * A[p].dwm);
    const Ax& q = A[(p + 1) % 3];
    const Ax& r = A[(p + 2) % 3];
    dG[p] = (fmaf(q.dw0, r.w0, W0 * r.dw0)) - (fmaf(q.dS, r.S, Tr * r.dS));
  }
  const float dR = fmaf(A[0].dw0, A[1].w0 * A[2].w0, W0 * fmaf(A[1].dw0, A[2].w0, W0 * A[2].dw0)) +
                   fmaf(A[0].dS, A[1].S * A[2].S, Tr * fmaf(A[1].dS, A[2].S, Tr * A[2].dS));
  f[0] = fmaf(dr, R0, rho * dR);
#pragma unroll
  for (int i = 1; i < Q19; ++i) {
    if (NNZ(i) == 1) {
      const int p = DX(i) ? 0 : (DY(i) ? 1 : 2);
      const float P_ = DC(i, p) > 0 ? Pp[p] : Pm[p];
      f[i] = fmaf(P_, G0, (P_ + rr * Wpm) * dG[p]);
    } else {
      const int p = DX(i) ? 0 : 1;
      const int q = DZ(i) ? 2 : 1;
      const float P_ = DC(i, p) > 0 ? Pp[p] : Pm[p];
      const float dwq = DC(i, q) > 0 ? A[q].dwp : A[q].dwm;
      f[i] = fmaf(P_, Wpm, (P_ + rr * Wpm) * dwq);
    }
  }
}

// Rest-equilibrium weight f^eq_i(1, 0, T) of the folded lattice.
__device__ __forceinline__ float wrest3(int i, float T) {
  const int nz = NNZ(i);
  if (nz == 0) return (1.f - T) * (1.f - T) * (1.f - T) + T * T * T;
  if (nz == 1) return 0.5f * T * (1.f - 2.f * T);
  return 0.25f * T * T;
}
// wrest3(i, Tr + d) - wrest3(i, Tr) for the emitted (non-rest) directions, formed from the
// deviation d: axis links 1/2 d (1 - 4 Tr - 2 d), face diagonals 1/4 d (2 Tr + d).
__device__ __forceinline__ float dwrest3(int i, float Tr, float d) {
  return NNZ(i) == 1 ? 0.5f * d * fmaf(-2.f, d, fmaf(-4.f, Tr, 1.f)) : 0.25f * d * fmaf(2.f, Tr, d);
}

__device__ __forceinline__ double block_sum3(double v, double* sh) {
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

// ---------------------------------------------------------------------------------------
// Gas node: pull, moments, energy-correction divergence, collision (MODE 0), the
// pre-collision moments only (MODE 1), or the moment field of the current step (MODE 2:
// dTg and K_j into Fdst with ghost copies; written by a pass over all gas nodes before
// the step, read by MODE 0 and 1 through Fsrc: reading R8 at the current time level).
// ---------------------------------------------------------------------------------------
template <class PT, int NS, bool PHI, int MODE, bool DET = false>
__device__ __forceinline__ void gas_node3(const DevParams& P, const PT* __restrict__ src, PT* __restrict__ dst,
                                          const uint64_t* __restrict__ code, int k, int aux,
                                          const float* __restrict__ Fsrc, float* __restrict__ Fdst,
                                          float* __restrict__ mom, float* __restrict__ Tgas, int* __restrict__ flags,
                                          float* __restrict__ s_h, int tid, uint32_t step, Acct* ac = nullptr) {
  const uint64_t cw = __ldg(code + k);
  const uint32_t seed = sizeof(PT) == 4 ? 0U : node_seed(k, step);
  const int n = aux & GAS_AUX_N;
  const int pl = (int)P.plane;
  const float Tr = P.Tref;
  const float ec0 = -3.f * Tr, ec1 = 1.f - 3.f * Tr, ec2 = 2.f - 3.f * Tr;
  float dr[NS], ax[NS], ay[NS], az[NS], ee[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const float v = pop_ld(src + (j * Q19) * pl + k, P.hsi[j]);
    if (MODE == 0) s_h[(j * Q19) * G3 + tid] = v;
    dr[j] = v;
    ax[j] = ay[j] = az[j] = 0.f;
    ee[j] = ec0 * v;
  }
  // Pull every direction (a rolled loop: the direction's components come from a table,
  // which keeps the code small); the loads of all species of one direction first.
#pragma unroll 1
  for (int i = 1; i < Q19; ++i) {
    const int4 e = c3_e[i];  // {ex, ey, ez, ecoef index}
    const int off = e.x + e.y * P.pitch + e.z * (int)P.slab;
    const uint32_t st = stencil_of3(cw, i);
    const float4 cp = c3_p[st];
    const float2 cq = c3_q[st];
    const int2 cm = c3_m[st];
    const int dA = cm.x * off, dB = cm.y * off;
    float v1[NS], vA[NS], vB[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const int b = (j * Q19 + i) * pl + k;
      v1[j] = pop_ld(src + (b - off), P.hsi[j]);
      vA[j] = vB[j] = 0.f;
      if (!P.onlattice[j]) {
        vA[j] = pop_ld(src + (b + dA), P.hsi[j]);
        vB[j] = pop_ld(src + (b + dB), P.hsi[j]);
      }
    }
    const float ec = e.w == 1 ? ec1 : ec2;
    const float fx = float(e.x), fy = float(e.y), fz = float(e.z);
    // exact accounts: classes of the node s1 comes from and of the node this node's own
    // population i streams into
    uint32_t cu = GAS, cd = GAS;
    if constexpr (DET) {
      cu = node_class3(__ldg(code + k - off));
      cd = node_class3(__ldg(code + k + off));
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
        const double ew = eps_weight(P, j, e.w);
        ac->dint += ew * (double(v) - double(v1[j]));
        const double off0 = double(P.rref[j]) * double(P.W0_19[i]);
        if (cu == INLET) ac->qin += ew * (double(v1[j]) + off0);
        if (cu == OUTLET) ac->qout += ew * (double(v1[j]) + off0);
        if (cd == INLET || cd == OUTLET) {
          const double own = ew * (double(pop_ld(src + ((j * Q19 + i) * pl + k), P.hsi[j])) + off0);
          if (cd == INLET) ac->qin -= own;
          else ac->qout -= own;
        }
      }
      if (MODE == 0) s_h[(j * Q19 + i) * G3 + tid] = v;
      dr[j] += v;
      ax[j] = fmaf(fx, v, ax[j]);
      ay[j] = fmaf(fy, v, ay[j]);
      az[j] = fmaf(fz, v, az[j]);
      ee[j] = fmaf(ec, v, ee[j]);
    }
  }
  // Mixture moments (Eq. moments_of_g, Eq. moments_of_f), deviation form.
  float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, C = 0.f, de = 0.f;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const float rho = P.rref[j] + dr[j];
    r += rho;
    jx = fmaf(P.c[j], ax[j], jx);
    jy = fmaf(P.c[j], ay[j], jy);
    jz = fmaf(P.c[j], az[j], jz);
    C = fmaf(rho, P.invM[j], C);
    de = fmaf(P.c2[j], ee[j], de);
  }
  const float dTg = (de - (jx * jx + jy * jy + jz * jz) / r) * (1.f / 3.f) / C;
  if (MODE == 2) {
    const bool gh = (aux & GAS_AUX_GHOST) != 0;
    Ghost3 g{{0, 0, 0}};
    if (gh) {
      int x = 0, y = 0, z = 0;
      xyz_of(P, n, x, y, z);
      g = ghost3(P, x, y, z);
    }
    store3(Fdst, k, g, gh, dTg);
#pragma unroll
    for (int j = 0; j < NS; ++j)
      store3(Fdst + (long long)(1 + j) * pl, k, g, gh, P.kcoef[j] * ((P.rref[j] + dr[j]) * P.invM[j]) * (Tr + dTg));
    return;
  }
  // Energy-correction divergence from the moment field of this step on the 6 axis
  // neighbours (faces to non-gas nodes carry no flux).
  float divq[NS];
  float sdq = 0.f;
#pragma unroll
  for (int j = 0; j < NS; ++j) divq[j] = 0.f;
  if (PHI) {
    const float Tc = __ldg(Fsrc + k);
#pragma unroll
    for (int d = 1; d <= 6; ++d) {
      if (!((cw >> (NBR_SHIFT3 + d - 1)) & 1ull)) continue;
      const int kn = k + (int)poff(P, d);
      const float dTn = __ldg(Fsrc + kn) - Tc;
#pragma unroll
      for (int j = 0; j < NS; ++j)
        divq[j] = fmaf(0.5f * (__ldg(Fsrc + (long long)(1 + j) * pl + k) + __ldg(Fsrc + (long long)(1 + j) * pl + kn)),
                       dTn, divq[j]);
    }
#pragma unroll
    for (int j = 0; j < NS; ++j) sdq += divq[j];
  }
  const float ux = jx / r, uy = jy / r, uz = jz / r;
  const float dT = dTg + sdq / (6.f * C);
  const float T = Tr + dT;
  if (MODE == 1) {
#pragma unroll
    for (int j = 0; j < NS; ++j) mom[(long long)j * P.n + n] = P.rref[j] + dr[j];
    mom[(long long)NS * P.n + n] = ux;
    mom[(long long)(NS + 1) * P.n + n] = uy;
    mom[(long long)(NS + 2) * P.n + n] = uz;
    mom[(long long)(NS + 3) * P.n + n] = dT;  // T - T_ref
    return;
  }
  const bool gh = (aux & GAS_AUX_GHOST) != 0;
  Ghost3 g{{0, 0, 0}};
  int x = 0, y = 0, z = 0;
  if (gh || (aux & GAS_AUX_OUTLET)) xyz_of(P, n, x, y, z);
  if (gh) g = ghost3(P, x, y, z);
  if (Tgas != nullptr) Tgas[n] = dT;  // T - T_ref
  if (!(r > 0.f) || !(T > 0.f) || !isfinite(ux + uy + uz + T)) atomicOr(flags, 1);

  // Corrective diffusion velocity (reading R3).
  float ncx = 0.f, ncy = 0.f, ncz = 0.f, den = 0.f;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const float rho = P.rref[j] + dr[j];
    ncx = fmaf(P.uc_w[j], fmaf(P.c[j], ax[j], -rho * ux), ncx);
    ncy = fmaf(P.uc_w[j], fmaf(P.c[j], ay[j], -rho * uy), ncy);
    ncz = fmaf(P.uc_w[j], fmaf(P.c[j], az[j], -rho * uz), ncz);
    den = fmaf(P.uc_w[j], rho, den);
  }
  const float iden = 1.f / den;
  const float Uc[3] = {ncx * iden, ncy * iden, ncz * iden};
  const float u[3] = {ux, uy, uz};

  float* s_m = s_h + NS * Q19 * G3;
#pragma unroll
  for (int j = 0; j < NS; ++j) s_m[j * G3 + tid] = divq[j];
#pragma unroll 1
  for (int j = 0; j < NS; ++j) {
    float drj = 0.f, Jj[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < Q19; ++i) {
      const float h = s_h[(j * Q19 + i) * G3 + tid];
      drj += h;
      if (DX(i)) Jj[0] += DX(i) > 0 ? h : -h;
      if (DY(i)) Jj[1] += DY(i) > 0 ? h : -h;
      if (DZ(i)) Jj[2] += DZ(i) > 0 ? h : -h;
    }
    const float rr = P.rref[j];
    const float rho = rr + drj;
    const float M = P.M[j], sM = P.sqrtM[j];
    // f-momentum (Eq. moments_of_g) and the species velocity of f*, limited for trace
    // species (reading R15).
    float uj[3] = {ux, uy, uz};
    if (rho != 0.f) {
      const float ir = 1.f / rho;
      const float lim2 = fmaxf(1.f - T, 0.f) * P.invM[j];
      bool big = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        // u + (J_j - rho_j u + a2 rho_j U^c) / ((1 + a2) rho_j): formed from the diffusion
        // flux, so that no rounded constant multiplies rho_j u: the direct form leaves a
        // momentum source ~1e-7 rho_j u per collision, a velocity error that builds up
        const float Dj = fmaf(-rho, u[a], P.c[j] * Jj[a]);
        uj[a] = fmaf(fmaf(P.a2[j] * rho, Uc[a], Dj) * P.inv1a2[j], ir, u[a]);
        big |= uj[a] * uj[a] > lim2;
      }
      if (big) {
        const float lim = sqrtf(lim2);
#pragma unroll
        for (int a = 0; a < 3; ++a) uj[a] = fminf(fmaxf(uj[a], -lim), lim);
      }
    }
    Ax Ae[3], As[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Ae[a] = axis3(sM, P.sqrtM_lo[j], M, u[a], T, dT);
      As[a] = axis3(sM, P.sqrtM_lo[j], M, uj[a], T, dT);
    }
    float feq[Q19], fst[Q19];
    feq_dev3(drj, rr, Tr, Ae, feq);
    feq_dev3(drj, rr, Tr, As, fst);
    const float om = P.omega[j], omt = P.omega[j] * P.t1t2[j];
    // w1 tau1 Psi_i = sum_a (8 c_j psi_ia) gf_a, gf_a = w1 tau1 rho U^c_a / (8 c_j tau2)
    const float gfs = P.wt1[j] * rho * P.invtau2[j] * 0.125f * sM;
    const float gf[3] = {gfs * Uc[0], gfs * Uc[1], gfs * Uc[2]};
    // w1 tau1 Phi_i with phi = M_j {-1, 1/6 on the axis links, 0 on diagonals}
    const float gphi = P.wt1[j] * M * s_m[j * G3 + tid];
    PT* out = dst + (long long)j * Q19 * pl;
    const float sc = P.hs[j];
#pragma unroll
    for (int i = 0; i < Q19; ++i) {
      float force = 0.f;
      if (NNZ(i) == 0) force = -gphi;
      if (NNZ(i) == 1) {
        const int p = DX(i) ? 0 : (DY(i) ? 1 : 2);
        force = fmaf(8.f * DC(i, p), gf[p], gphi * (1.f / 6.f));
      }
      if (NNZ(i) == 2) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (DC(i, a)) force = fmaf(-float(DC(i, a)), gf[a], force);
      }
      const float h = s_h[(j * Q19 + i) * G3 + tid];
      const float hn = fmaf(-om, h - fst[i], fmaf(-omt, fst[i] - feq[i], h + force));
      pop_store3(out + (long long)i * pl, k, g, gh, hn, sc, seed, j * Q19 + i);
      if constexpr (DET)  // FP32 storage: hn is the value stored
        if (i > 0) ac->dcol += eps_weight(P, j, NNZ(i)) * (double(hn) - double(h));
    }
  }

  // Outlet (reading R13): equilibrium at the outlet pressure with this node's
  // composition, velocity and temperature, written into the +x neighbour.
  if (aux & GAS_AUX_OUTLET) {
    const float Cout = P.p_out / T;
    Ghost3 go{{0, 0, 0}};
    const bool ogh = gh;
    if (ogh) go = ghost3(P, x + 1, y, z);
#pragma unroll 1
    for (int j = 0; j < NS; ++j) {
      const float rj = (P.rref[j] + dr[j]) * P.invM[j] / C * Cout * P.M[j];
      Ax Ae[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) Ae[a] = axis3(P.sqrtM[j], P.sqrtM_lo[j], P.M[j], u[a], T, dT);
      float f[Q19];
      feq_dev3(rj - P.rref[j], P.rref[j], Tr, Ae, f);
#pragma unroll
      for (int i = 0; i < Q19; ++i)
        pop_store3(dst + (long long)(j * Q19 + i) * pl, k + 1, go, ogh, f[i], P.hs[j], seed, NS * Q19 + j * Q19 + i);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Solid node: FD heat step (7-point); interface wall nodes also run the reactive
// diffusive wall (Sec. 4.3) and receive the reaction heat and the coupling.
// ---------------------------------------------------------------------------------------
template <int NS>
__device__ __forceinline__ void rates3(const DevParams& P, const float (&rw)[NS], const float* kr, float* rate) {
  float Cw[NS], Ct = 0.f;
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    Cw[j] = rw[j] * P.invM[j];
    Ct += Cw[j];
  }
  const float iCt = 1.f / Ct;
  for (int q = 0; q < P.nr; ++q) {
    float fwd = 1.f, bwd = 1.f;
    const bool conc = P.rate_form[q] == FDLBM_RATE_CONC_BILINEAR;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const float v = conc ? Cw[j] : Cw[j] * iCt;
      const int nu = P.nu[q][j];
      for (int m = 0; m < -nu; ++m) fwd *= v;
      for (int m = 0; m < nu; ++m) bwd *= v;
    }
    rate[q] = conc ? kr[q] * fwd : kr[q] * (fwd - bwd * P.inv_Keq[q]);
  }
}

template <class PT, int NS, bool DET = false>
__device__ __forceinline__ void solid_node3(const DevParams& P, const PT* __restrict__ src, PT* __restrict__ dst,
                                            const float* __restrict__ Ts_src, float* __restrict__ Ts_dst,
                                            const uint64_t* __restrict__ code, const float* __restrict__ Tgas, int n,
                                            double (&acc)[LG_COUNT], float* __restrict__ rw_prev, int idx,
                                            uint32_t step) {
  int x, y, z;
  xyz_of(P, n, x, y, z);
  const int k = pad3(P, x, y, z);
  const uint64_t cw = __ldg(code + k);
  const float Tx = Ts_src[n];
  float lap = 0.f, gas_term = 0.f;
#pragma unroll
  for (int d = 1; d <= 6; ++d) {
    const int nb = lat3(P, x + DX(d), y + DY(d), z + DZ(d));
    if ((cw >> (NBR_SHIFT3 + d - 1)) & 1ull) {
      lap += Ts_src[nb] - Tx;
      continue;
    }
    if (nb < 0) {
      const int face = 2 * ((d - 1) / 2) + ((d & 1) ? 1 : 0);  // +x -> x+ (1), -x -> x- (0), ...
      if (P.fixedT_face[face]) {
        lap += P.dTout - Tx;
        acc[LG_QFIXEDT] += double(P.rhocp_s) * double(P.alpha_s) * double(P.dTout - Tx);
      }
      continue;
    }
    if (Tgas != nullptr && node_class3(__ldg(code + k + (int)poff(P, d))) == GAS) gas_term += Tgas[nb] - Tx;
  }
  float Tn = fmaf(P.alpha_s, lap, Tx);
  if (node_class3(cw) == WALL) {
    const int pl = (int)P.plane;
    const float Tw = P.Tref + Tx;
    uint32_t arr = 0;
    for (int i = 1; i < Q19; ++i)
      if (stencil_of3(cw, i) != ST_NOT_ARRIVAL) arr |= 1u << i;
    // emitted shape W0_i + dW_i at the wall temperature; dW from the deviation Tx
    float B = 0.f, dB = 0.f;
    for (int i = 1; i < Q19; ++i)
      if (arr & (1u << OPP3(i))) {
        B += wrest3(i, Tw);
        dB += dwrest3(i, P.Tref, Tx);
      }
    float A[NS], Ah[NS], rw[NS], mj[NS];
    float Earr = 0.f, W0arr = 0.f;
#pragma unroll
    for (int j = 0; j < NS; ++j) Ah[j] = 0.f;
#pragma unroll 1
    for (int i = 1; i < Q19; ++i) {
      if (!(arr & (1u << i))) continue;
      const int off = DX(i) + DY(i) * P.pitch + DZ(i) * (int)P.slab;
      const uint32_t st = stencil_of3(cw, i);
      const float4 cp = c3_p[st];
      const float2 cq = c3_q[st];
      const int2 cm = c3_m[st];
      const int dA = cm.x * off, dB = cm.y * off;
      const float e2h = 0.5f * float(DX(i) * DX(i) + DY(i) * DY(i) + DZ(i) * DZ(i));
      W0arr += P.W0_19[i];
      float v1[NS], vA[NS], vB[NS];
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const int b = (j * Q19 + i) * pl + k;
        v1[j] = pop_ld(src + (b - off), P.hsi[j]);
        vA[j] = pop_ld(src + (b + dA), P.hsi[j]);
        vB[j] = pop_ld(src + (b + dB), P.hsi[j]);
      }
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        float v = v1[j];
        if (!P.onlattice[j]) {
          const float d1 = fmaf(-cp.z, v1[j], fmaf(cp.x, vA[j], cp.y * vB[j]));
          const float d2 = fmaf(-cq.y, v1[j], fmaf(cp.w, vA[j], cq.x * vB[j]));
          v = fmaf(P.ha[j], d1, fmaf(P.ha2[j], d2, v1[j]));
        }
        if constexpr (DET) {  // arrival's departure from the shift; its energy, exactly
          const double ew = eps_weight(P, j, DX(i) * DX(i) + DY(i) * DY(i) + DZ(i) * DZ(i));
          acc[LG_DINT] += ew * (double(v) - double(v1[j]));
          acc[LG_QWALLX] -= ew * (double(v) + double(P.rref[j]) * double(P.W0_19[i]));
        }
        Ah[j] += v;  // deviations; the rest part rref W0 is added below
        Earr = fmaf(e2h * P.c2[j], v, Earr);
      }
    }
    const float iB = 1.f / B;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      A[j] = fmaf(P.rref[j], W0arr, Ah[j]);
      rw[j] = A[j] * iB;
      mj[j] = 0.f;
    }
    float rate[MAX_NR] = {0.f, 0.f, 0.f, 0.f};
    const bool cat = (cw & CATALYTIC_BIT) && P.nr > 0;
    if (cat) {
      float kr[MAX_NR];
      const float TK = P.T3T0 * Tw;
      for (int q = 0; q < P.nr; ++q) kr[q] = P.k0[q] * expf(-P.EaR[q] / TK);
      float* rp = rw_prev + idx;
      if (rp[0] == rp[0]) {
#pragma unroll
        for (int j = 0; j < NS; ++j) rw[j] = rp[(long long)j * P.n_wall_list];
      }
      bool conv = false;
      for (int it = 0; it < P.rho_w_maxit; ++it) {
        rates3<NS>(P, rw, kr, rate);
        float dmax = 0.f, rmax = 0.f;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          float mm = 0.f;
          for (int q = 0; q < P.nr; ++q) mm += P.M[j] * float(P.nu[q][j]) * rate[q];
          const float nw = (A[j] + mm) * iB;
          dmax = fmaxf(dmax, fabsf(nw - rw[j]));
          rmax = fmaxf(rmax, fabsf(nw));
          rw[j] = nw;
        }
        if (dmax <= fmaxf(P.rho_w_tol, 4.f * FLT_EPSILON * rmax)) {
          conv = true;
          break;
        }
      }
      if (!conv) acc[LG_NOCONV] += 1.0;
#pragma unroll
      for (int j = 0; j < NS; ++j) rp[(long long)j * P.n_wall_list] = rw[j];
      rates3<NS>(P, rw, kr, rate);
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        float mm = 0.f;
        for (int q = 0; q < P.nr; ++q) mm += P.M[j] * float(P.nu[q][j]) * rate[q];
        mj[j] = mm;
      }
    }
    const Ghost3 g = ghost3(P, x, y, z);
    const bool gh = g.d[0] || g.d[1] || g.d[2];
    const uint32_t seed = sizeof(PT) == 4 ? 0U : node_seed(k, step);
    float Eout = 0.f;
    // emitted deviation dscale W0_i + (rref + dscale) dW_i, dscale = (A + m) / B - rref
    // = (sum of arrived deviations - rref dB + m) / B (the rest parts of the mirrored
    // arrival and emission sets cancel)
    float dsc[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) dsc[j] = (fmaf(-P.rref[j], dB, Ah[j]) + mj[j]) * iB;
#pragma unroll 1
    for (int i = 1; i < Q19; ++i) {
      if (!(arr & (1u << OPP3(i)))) continue;
      const float dwr = dwrest3(i, P.Tref, Tx);
      const float e2h = 0.5f * float(DX(i) * DX(i) + DY(i) * DY(i) + DZ(i) * DZ(i));
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const float dv = fmaf(dsc[j], P.W0_19[i], (P.rref[j] + dsc[j]) * dwr);
        pop_store3(dst + (long long)(j * Q19 + i) * pl, k, g, gh, dv, P.hs[j], seed, j * Q19 + i);
        if constexpr (DET)  // FP32 storage: dv is the value stored
          acc[LG_QWALLX] += eps_weight(P, j, DX(i) * DX(i) + DY(i) * DY(i) + DZ(i) * DZ(i)) *
                            (double(dv) + double(P.rref[j]) * double(P.W0_19[i]));
        Eout = fmaf(e2h * P.c2[j], dv, Eout);
      }
    }
    float q = 0.f;
    if (cat)
      for (int r = 0; r < P.nr; ++r) q += P.heat[r] * rate[r];
    const float dE = Eout - Earr;
    const float couple = P.coupling == FDLBM_COUPLING_PAPER ? P.kappa_f * gas_term : -dE;
    Tn += (q + couple) * P.inv_rhocp_s;
    acc[LG_QRXN] += q;
    acc[LG_QWALL] += dE;
    acc[LG_QCOUPLE] += couple;
  }
  Ts_dst[n] = Tn;
  if constexpr (DET) acc[LG_DH] += double(P.rhocp_s) * (double(Tn) - double(Tx));
}

template <int NQ = LG_BASIC>
__device__ __forceinline__ void ledger_store3(double (&acc)[LG_COUNT], double* __restrict__ slot) {
  __shared__ double sh[NQ][G3 / 32];
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

// One time step in one launch (blocks: {role 0 gas / 1 solid, first, count, 0}).
template <class PT, int NS, bool PHI, bool DET = false>
__global__ void __launch_bounds__(G3, 4) step_kernel3(
    DevParams P, const PT* __restrict__ src, PT* __restrict__ dst, const uint64_t* __restrict__ code,
    const int2* __restrict__ gas_list, const int32_t* __restrict__ solid_list, const int4* __restrict__ blocks,
    const float* __restrict__ Fsrc, float* __restrict__ Fdst, const float* __restrict__ Ts_src,
    float* __restrict__ Ts_dst, const float* __restrict__ Tgas_src, float* __restrict__ Tgas_dst,
    double* __restrict__ ledger, int* __restrict__ flags, float* __restrict__ rw_prev, uint32_t step) {
  extern __shared__ float smem[];
  const int4 d = __ldg(blocks + blockIdx.x);
  const int tid = threadIdx.x;
  if (d.x == 0) {
    if constexpr (DET) {
      Acct ac{0.0, 0.0, 0.0, 0.0};
      if (tid < d.z) {
        const int2 g = __ldg(gas_list + d.y + tid);
        gas_node3<PT, NS, PHI, 0, true>(P, src, dst, code, g.x, g.y, Fsrc, Fdst, nullptr, Tgas_dst, flags, smem, tid,
                                        step, &ac);
      }
      double acc[LG_COUNT];
#pragma unroll
      for (int q = 0; q < LG_COUNT; ++q) acc[q] = 0.0;
      acc[LG_QIN] = ac.qin;
      acc[LG_QOUT] = ac.qout;
      acc[LG_DINT] = ac.dint;
      acc[LG_DCOL] = ac.dcol;
      ledger_store3<LG_COUNT>(acc, ledger + (long long)blockIdx.x * LG_COUNT);
    } else if (tid < d.z) {
      const int2 g = __ldg(gas_list + d.y + tid);
      gas_node3<PT, NS, PHI, 0>(P, src, dst, code, g.x, g.y, Fsrc, Fdst, nullptr, Tgas_dst, flags, smem, tid, step);
    }
    return;
  }
  double acc[LG_COUNT];
#pragma unroll
  for (int q = 0; q < LG_COUNT; ++q) acc[q] = 0.0;
  if (tid < d.z)
    solid_node3<PT, NS, DET>(P, src, dst, Ts_src, Ts_dst, code, Tgas_src, __ldg(solid_list + d.y + tid), acc, rw_prev,
                             d.y + tid, step);
  ledger_store3<DET ? LG_COUNT : LG_BASIC>(acc, ledger + (long long)blockIdx.x * LG_COUNT);
}

// A pass over every gas node: MODE 1, the pre-collision moments of the step that reads
// src (rho_j, ux, uy, uz, T into mom); MODE 2, that step's moment field (into Fdst).
template <class PT, int NS, bool PHI, int MODE>
__global__ void __launch_bounds__(G3) gas_pass_kernel3(DevParams P, const PT* __restrict__ src,
                                                      const uint64_t* __restrict__ code,
                                                      const int2* __restrict__ gas_list,
                                                      const float* __restrict__ Fsrc, float* __restrict__ Fdst,
                                                      float* __restrict__ mom) {
  extern __shared__ float smem[];
  const int t = blockIdx.x * G3 + threadIdx.x;
  if (t >= P.n_gas) return;
  const int2 g = __ldg(gas_list + t);
  gas_node3<PT, NS, PHI, MODE>(P, src, nullptr, code, g.x, g.y, Fsrc, Fdst, mom, nullptr, nullptr, smem, threadIdx.x,
                               0U);
}

template <int NS>
constexpr size_t smem3() {
  return sizeof(float) * (size_t)(NS * Q19 + NS) * G3;
}

// ---------------------------------------------------------------------------------------
// Initialisation over every padded cell (FP64 arithmetic, then rounded), so that ghost
// copies start consistent.
// ---------------------------------------------------------------------------------------
__device__ double wf_d(int e, double v, double M, double T) {
  return e == 0 ? 1.0 - M * v * v - T : 0.5 * (double(e) * sqrt(M) * v + M * v * v + T);
}
// Folded equilibrium of direction i (closed form of the fold, FP64).
__device__ double feq3_d(int i, double rho, const double (&u)[3], double M, double T) {
  const int e[3] = {DX(i), DY(i), DZ(i)};
  const int nz = NNZ(i);
  double w0[3], S[3];
  for (int a = 0; a < 3; ++a) {
    w0[a] = wf_d(0, u[a], M, T);
    S[a] = M * u[a] * u[a] + T;
  }
  if (nz == 0) return rho * (w0[0] * w0[1] * w0[2] + S[0] * S[1] * S[2]);
  if (nz == 1) {
    const int p = e[0] ? 0 : (e[1] ? 1 : 2);
    const int q = (p + 1) % 3, r = (p + 2) % 3;
    return rho * wf_d(e[p], u[p], M, T) * (w0[q] * w0[r] - S[q] * S[r]);
  }
  double f = rho;
  for (int a = 0; a < 3; ++a)
    if (e[a]) f *= wf_d(e[a], u[a], M, T);
  return f;
}

template <class PT>
__global__ void init_kernel3(DevParams P, PT* __restrict__ h0, PT* __restrict__ h1, float* __restrict__ Ts0,
                             float* __restrict__ Ts1, float* __restrict__ F0, float* __restrict__ F1,
                             float* __restrict__ mom, float* __restrict__ Tgas, const uint64_t* __restrict__ code,
                             const double* __restrict__ X, const double* __restrict__ u, const double* __restrict__ Tl,
                             const double* __restrict__ Tsl, const double* __restrict__ Cn,
                             const double* __restrict__ inlet) {
  const long long cells = P.slab * (P.nz + 2 * P.zoff);
  for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < cells;
       kk += (long long)gridDim.x * blockDim.x) {
    const int k = (int)kk;
    int px = k % P.pitch, py = (k / P.pitch) % (P.ny + 2 * P.yoff), pz = (int)(kk / P.slab);
    int x = px - P.xoff, y = py - P.yoff, z = pz - P.zoff;
    bool inside = true;
    if (x < 0 || x >= P.nx) {
      if (!P.periodic_x || x < -GHOST3 || x >= P.nx + GHOST3) inside = false;
      else x = x < 0 ? x + P.nx : x - P.nx;
    }
    if (y < 0 || y >= P.ny) {
      if (!P.periodic_y || y < -GHOST3 || y >= P.ny + GHOST3) inside = false;
      else y = y < 0 ? y + P.ny : y - P.ny;
    }
    if (z < 0 || z >= P.nz) {
      if (!P.periodic_z || z < -GHOST3 || z >= P.nz + GHOST3) inside = false;
      else z = z < 0 ? z + P.nz : z - P.nz;
    }
    if (!inside) continue;
    const bool real = px - P.xoff == x && py - P.yoff == y && pz - P.zoff == z;
    const int n = x + P.nx * (y + P.ny * z);
    const uint64_t cw = code[pad3(P, x, y, z)];
    const uint32_t c = node_class3(cw);
    const double Tref = P.Tref;
    double Xn[MAX_NS];
    for (int j = 0; j < P.ns; ++j) Xn[j] = X[(long long)j * P.n + n];
    double uu[3] = {u[n], u[P.n + n], u[2LL * P.n + n]};
    double T = Tl[n], C = Cn[n];
    if (c == INLET) {
      for (int j = 0; j < P.ns; ++j) Xn[j] = inlet[j];
      uu[0] = inlet[P.ns + 1];
      uu[1] = uu[2] = 0.0;
      T = inlet[P.ns];
      C = 1.0;
    }
    const double z0[3] = {0.0, 0.0, 0.0};
    if (c == GAS || c == INLET || c == OUTLET) {
      for (int j = 0; j < P.ns; ++j) {
        const double M = P.M[j];
        const double rho = C * Xn[j] * M;
        for (int i = 0; i < Q19; ++i) {
          const double v = feq3_d(i, rho, uu, M, T) - double(P.rref[j]) * feq3_d(i, 1.0, z0, 1.0, Tref);
          h0[(long long)(j * Q19 + i) * P.plane + k] = h1[(long long)(j * Q19 + i) * P.plane + k] =
              pop_enc<PT>(float(v), P.hs[j]);
        }
      }
      if (c == GAS) {
        F0[k] = F1[k] = float(T - Tref);
        for (int j = 0; j < P.ns; ++j)
          F0[(long long)(1 + j) * P.plane + k] = F1[(long long)(1 + j) * P.plane + k] =
              float(double(P.kcoef[j]) * C * Xn[j] * T);
      }
      if (c == GAS && real) {
        for (int j = 0; j < P.ns; ++j) mom[(long long)j * P.n + n] = float(C * Xn[j] * P.M[j]);
        for (int a = 0; a < 3; ++a) mom[(long long)(P.ns + a) * P.n + n] = float(uu[a]);
        mom[(long long)(P.ns + 3) * P.n + n] = float(T - double(P.Tref));
        Tgas[n] = Tgas[P.n + n] = float(T - double(P.Tref));
      }
    } else if (c == WALL || c == SOLID) {
      const double Ts = Tsl[n];
      if (real) Ts0[n] = Ts1[n] = float(Ts - Tref);
      if (c == WALL)
        for (int j = 0; j < P.ns; ++j) {
          const double rho = C * Xn[j] * P.M[j];
          for (int i = 1; i < Q19; ++i) {
            if (stencil_of3(cw, OPP3(i)) == ST_NOT_ARRIVAL) continue;
            const double v = rho * feq3_d(i, 1.0, z0, 1.0, Ts) - double(P.rref[j]) * feq3_d(i, 1.0, z0, 1.0, Tref);
            h0[(long long)(j * Q19 + i) * P.plane + k] = h1[(long long)(j * Q19 + i) * P.plane + k] =
                pop_enc<PT>(float(v), P.hs[j]);
          }
        }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Outputs and reductions
// ---------------------------------------------------------------------------------------
// T and T_s in kelvin, or with dev as deviations from the inlet temperature (kelvin).
__global__ void moments_out_kernel3(DevParams P, const float* __restrict__ mom, const float* __restrict__ Ts,
                                    const uint64_t* __restrict__ code, float* __restrict__ dst, int dev) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P.n) return;
  int x, y, z;
  xyz_of(P, n, x, y, z);
  const uint32_t c = node_class3(code[pad3(P, x, y, z)]);
  const int ns = P.ns;
  const long long N = P.n;
  for (int f = 0; f < 2 * ns + 5; ++f) dst[f * N + n] = 0.f;
  if (c == GAS) {
    float C = 0.f;
    for (int j = 0; j < ns; ++j) C += mom[j * N + n] * P.invM[j];
    for (int j = 0; j < ns; ++j) {
      dst[j * N + n] = mom[j * N + n];
      dst[(ns + j) * N + n] = mom[j * N + n] * P.invM[j] / C;
    }
    for (int a = 0; a < 3; ++a) dst[(2 * ns + a) * N + n] = mom[(ns + a) * N + n];
    dst[(2 * ns + 3) * N + n] = (dev ? mom[(ns + 3) * N + n] + P.Tdev_off : P.Tref + mom[(ns + 3) * N + n]) * P.T3T0;
  } else if (c == WALL || c == SOLID) {
    dst[(2 * ns + 4) * N + n] = (dev ? Ts[n] + P.Tdev_off : P.Tref + Ts[n]) * P.T3T0;
  }
}

template <class PT>
__global__ void populations_out_kernel3(DevParams P, const PT* __restrict__ h, float* __restrict__ dst) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)P.ns * Q19 * P.n;
  if (q >= total) return;
  const int n = int(q % P.n);
  const int ji = int(q / P.n);
  const int i = ji % Q19, j = ji / Q19;
  int x, y, z;
  xyz_of(P, n, x, y, z);
  dst[q] = pop_ld(h + ((long long)ji * P.plane + pad3(P, x, y, z)), P.hsi[j]) + P.rref[j] * P.W0_19[i];
}

// E_gas (f-moments + in-transit wall emissions), H_solid, mass_j, moles_j.
template <class PT>
__global__ void totals_kernel3(DevParams P, const float* __restrict__ mom, const PT* __restrict__ h,
                               const float* __restrict__ Ts, const uint64_t* __restrict__ code,
                               double* __restrict__ out) {
  __shared__ double sh[8];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int ns = P.ns;
  const long long N = P.n;
  double E = 0.0, H = 0.0, mass[MAX_NS], moles[MAX_NS];
  for (int j = 0; j < ns; ++j) mass[j] = moles[j] = 0.0;
  if (n < P.n) {
    int x, y, z;
    xyz_of(P, n, x, y, z);
    const int k = pad3(P, x, y, z);
    const uint64_t cw = code[k];
    const uint32_t c = node_class3(cw);
    if (c == GAS) {
      double C = 0.0, r = 0.0, u2 = 0.0;
      for (int j = 0; j < ns; ++j) {
        const double rj = mom[j * N + n];
        mass[j] = rj;
        moles[j] = rj * double(P.invM[j]);
        C += rj / double(P.M[j]);
        r += rj;
      }
      for (int a = 0; a < 3; ++a) {
        const double v = mom[(ns + a) * N + n];
        u2 += v * v;
      }
      E = 1.5 * C * (double(P.Tref) + double(mom[(ns + 3) * N + n])) + 0.5 * r * u2;
    } else if (c == WALL || c == SOLID) {
      H = double(P.rhocp_s) * (double(P.Tref) + double(Ts[n]));
      if (c == WALL)
        for (int i = 1; i < Q19; ++i) {
          if (stencil_of3(cw, OPP3(i)) == ST_NOT_ARRIVAL) continue;
          for (int j = 0; j < ns; ++j) {
            const double w = double(pop_ld(h + ((long long)(j * Q19 + i) * P.plane + k), P.hsi[j])) +
                             double(P.rref[j]) * double(P.W0_19[i]);
            mass[j] += w;
            moles[j] += w / double(P.M[j]);
            E += 0.5 * double(P.c2[j]) * double(NNZ(i)) * w;
          }
        }
    }
  }
  double s = block_sum3(E, sh);
  if (threadIdx.x == 0) atomicAdd(out + 0, s);
  s = block_sum3(H, sh);
  if (threadIdx.x == 0) atomicAdd(out + 1, s);
  for (int j = 0; j < ns; ++j) {
    s = block_sum3(mass[j], sh);
    if (threadIdx.x == 0) atomicAdd(out + 2 + j, s);
    s = block_sum3(moles[j], sh);
    if (threadIdx.x == 0) atomicAdd(out + 2 + ns + j, s);
  }
}

// Residual sums over the fields ux, uy, uz, X_j, T (gas) and Ts (solid): sum (F - snap)^2
// and sum (F - ref)^2; then the snapshot is updated.
__global__ void residual_kernel3(DevParams P, const float* __restrict__ mom, const float* __restrict__ Ts,
                                 const uint64_t* __restrict__ code, float* __restrict__ snap,
                                 double* __restrict__ out) {
  __shared__ double sh[8];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int ns = P.ns, nf = ns + 5;
  const long long N = P.n;
  uint32_t c = OUTSIDE;
  if (n < P.n) {
    int x, y, z;
    xyz_of(P, n, x, y, z);
    c = node_class3(code[pad3(P, x, y, z)]);
  }
  float C = 0.f;
  if (c == GAS)
    for (int j = 0; j < ns; ++j) C += mom[j * N + n] * P.invM[j];
  for (int f = 0; f < nf; ++f) {
    double d2 = 0.0, r2 = 0.0;
    const bool solid_field = f == nf - 1;
    const bool on = solid_field ? (c == WALL || c == SOLID) : (c == GAS);
    if (on) {
      float v, ref;
      if (f < 3) {
        v = mom[(ns + f) * N + n];
        ref = 0.f;
      } else if (f < 3 + ns) {
        const int j = f - 3;
        v = mom[j * N + n] * P.invM[j] / C;
        ref = P.Xin[j];
      } else if (f == 3 + ns) {  // temperatures as deviations from T_ref
        v = mom[(ns + 3) * N + n];
        ref = -P.Tdev_off;
      } else {
        v = Ts[n];
        ref = -P.Tdev_off;
      }
      const float o = snap[f * N + n];
      d2 = double(v - o) * double(v - o);
      r2 = double(v - ref) * double(v - ref);
      snap[f * N + n] = v;
    }
    double s = block_sum3(d2, sh);
    if (threadIdx.x == 0) atomicAdd(out + 2 * f, s);
    s = block_sum3(r2, sh);
    if (threadIdx.x == 0) atomicAdd(out + 2 * f + 1, s);
  }
}

template <class K>
cudaError_t opt_in_smem3(K kernel, size_t smem, unsigned long long& configured) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && !(configured & (1ull << dev))) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured |= 1ull << dev;
  }
  return cudaSuccess;
}

// One step: with the energy correction, first the moment field of the step into F[0]
// (every gas node), then the step kernel (or the moments pass) reading it.
template <class PT, int NS, bool PHI, bool DET = false>
cudaError_t step3_launch(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st,
                         uint32_t step) {
  const size_t smem = smem3<NS>();
  static unsigned long long configured[3] = {0, 0, 0};
  const PT* hs = static_cast<const PT*>(S.h[src]);
  cudaError_t e;
  const int gas_grid = (P.n_gas + G3 - 1) / G3;
  // The field pass and the moments pass keep no pulled values (they return before any use
  // of shared memory): launched without dynamic shared memory, they run at the occupancy
  // their registers allow (32 warps per SM) instead of the step kernel's 16.
  if (PHI && P.n_gas > 0) {
    gas_pass_kernel3<PT, NS, PHI, 2><<<gas_grid, G3, 0, st>>>(P, hs, S.code64, S.gas_list, nullptr, S.F[0], nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (moments_only) {
    if (P.n_gas <= 0) return cudaSuccess;
    gas_pass_kernel3<PT, NS, PHI, 1><<<gas_grid, G3, 0, st>>>(P, hs, S.code64, S.gas_list, S.F[0], nullptr, S.mom);
    return cudaGetLastError();
  }
  if (P.n_blocks <= 0) return cudaSuccess;
  if ((e = opt_in_smem3(step_kernel3<PT, NS, PHI, DET>, smem, configured[0])) != cudaSuccess) return e;
  const int dstb = 1 - src;
  const bool paper = P.coupling == FDLBM_COUPLING_PAPER;
  step_kernel3<PT, NS, PHI, DET><<<P.n_blocks, G3, smem, st>>>(
      P, hs, static_cast<PT*>(S.h[dstb]), S.code64, S.gas_list, S.solid_list, S.blocks, S.F[0], nullptr,
      S.Ts[src], S.Ts[dstb], paper ? S.Tgas + (long long)src * P.n : nullptr,
      paper ? S.Tgas + (long long)dstb * P.n : nullptr, S.ledger, S.flags, S.rw, step);
  return cudaGetLastError();
}

template <class PT, int NS>
cudaError_t step3_ns(const DevParams& P, const DevState& S, int src, bool mo, cudaStream_t st, uint32_t step) {
  if constexpr (sizeof(PT) == 4) {
    if (P.ledger_detail && !mo) return launch_step3_detail(P, S, src, st, step);
  }
  return P.energy_correction ? step3_launch<PT, NS, true>(P, S, src, mo, st, step)
                             : step3_launch<PT, NS, false>(P, S, src, mo, st, step);
}

template <class PT>
cudaError_t step3_pt(const DevParams& P, const DevState& S, int src, bool mo, cudaStream_t st, uint32_t step) {
  switch (P.ns) {
    case 1: return step3_ns<PT, 1>(P, S, src, mo, st, step);
    case 2: return step3_ns<PT, 2>(P, S, src, mo, st, step);
    case 3: return step3_ns<PT, 3>(P, S, src, mo, st, step);
    case 4: return step3_ns<PT, 4>(P, S, src, mo, st, step);
    case 5: return step3_ns<PT, 5>(P, S, src, mo, st, step);
    case 6: return step3_ns<PT, 6>(P, S, src, mo, st, step);
    default: return cudaErrorInvalidValue;
  }
}

template <class PT>
cudaError_t init3_pt(const DevParams& P, const DevState& S, const double* X, const double* u, const double* T_lat,
                     const double* Ts_lat, const double* C, const double* inlet, cudaStream_t st) {
  const long long cells = P.slab * (P.nz + 2 * P.zoff);
  const int grid = (int)std::min<long long>((cells + 255) / 256, 152LL * 64);
  init_kernel3<PT><<<grid, 256, 0, st>>>(P, static_cast<PT*>(S.h[0]), static_cast<PT*>(S.h[1]), S.Ts[0], S.Ts[1],
                                         S.F[0], S.F[1], S.mom, S.Tgas, S.code64, X, u, T_lat, Ts_lat, C, inlet);
  return cudaGetLastError();
}

}  // namespace

// Storage-dependent entry points, instantiated once per storage type in its own
// translation unit (FDLBM3_STORAGE_ENTRY_POINTS).
template <class PT>
cudaError_t storage3_step(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st,
                          uint32_t step) {
  return step3_pt<PT>(P, S, src, moments_only, st, step);
}

template <class PT>
cudaError_t storage3_init(const DevParams& P, const DevState& S, const double* X, const double* u,
                          const double* T_lat, const double* Ts_lat, const double* C, const double* inlet,
                          cudaStream_t st) {
  return init3_pt<PT>(P, S, X, u, T_lat, Ts_lat, C, inlet, st);
}

template <class PT>
cudaError_t storage3_populations_out(const DevParams& P, const DevState& S, int cur, float* dst, cudaStream_t st) {
  const long long total = (long long)P.ns * Q19 * P.n;
  populations_out_kernel3<PT><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, static_cast<const PT*>(S.h[cur]), dst);
  return cudaGetLastError();
}

template <class PT>
cudaError_t storage3_totals(const DevParams& P, const DevState& S, int cur, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(S.red, 0, sizeof(double) * totals_count(P.ns), st);
  if (e != cudaSuccess) return e;
  totals_kernel3<PT><<<(P.n + 255) / 256, 256, 0, st>>>(P, S.mom, static_cast<const PT*>(S.h[cur]), S.Ts[cur],
                                                       S.code64, S.red);
  return cudaGetLastError();
}

}  // namespace fdlbm

#define FDLBM3_STORAGE_ENTRY_POINTS(PREFIX, PT)                                                                  \
  PREFIX template cudaError_t storage3_step<PT>(const DevParams&, const DevState&, int, bool, cudaStream_t,     \
                                               uint32_t);                                                       \
  PREFIX template cudaError_t storage3_init<PT>(const DevParams&, const DevState&, const double*, const double*, \
                                               const double*, const double*, const double*, const double*,      \
                                               cudaStream_t);                                                   \
  PREFIX template cudaError_t storage3_populations_out<PT>(const DevParams&, const DevState&, int, float*,       \
                                                          cudaStream_t);                                        \
  PREFIX template cudaError_t storage3_totals<PT>(const DevParams&, const DevState&, int, cudaStream_t);
