// Internal declarations shared by the host side (fdlbm_api.cu) and the kernels
// (fdlbm_kernels.cu) of the solver library. Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fdlbm.h"

namespace fdlbm {

constexpr int Q = 9;
// Ghost layers around the lattice on the padded population/code arrays: the deepest
// pull reaches 3 nodes upstream of a cell one node outside the tile's lattice range.
constexpr int GHOST = 4;
constexpr int XOFF = 8;  // padded column of x = 0 (keeps rows 32-byte aligned)
constexpr int YOFF = GHOST;
constexpr int MAX_NS = FDLBM_MAX_SPECIES;
constexpr int MAX_NR = FDLBM_MAX_REACTIONS;

// Node classes (bits 0..2 of the node code word).
enum NodeClass : uint32_t { GAS = 0, INLET = 1, OUTLET = 2, WALL = 3, SOLID = 4, OUTSIDE = 7 };
// Streaming stencils, 3 bits per direction i = 1..8 at bit 4 + 3 (i - 1).
enum Stencil : uint32_t { ST_NONE = 0, ST_CENTRAL = 1, ST_FORWARD = 2, ST_BACKWARD = 3,
                          ST_LIN_S0 = 4, ST_LIN_S2 = 5, ST_NOT_ARRIVAL = 7 };
constexpr uint32_t CATALYTIC_BIT = 1u << 3;
constexpr int STENCIL_SHIFT = 4;
// Bits 28..31: a gas node has a gas neighbour, a solid (wall or interior) node a solid
// neighbour, along direction 1..4 (+x, +y, -x, -y).
constexpr int NBR_GAS_SHIFT = 28;

__host__ __device__ inline uint32_t node_class(uint32_t code) { return code & 7u; }
__host__ __device__ inline uint32_t stencil_of(uint32_t code, int i) {
  return (code >> (STENCIL_SHIFT + 3 * (i - 1))) & 7u;
}

// Scalars every kernel needs, passed by value (kernel parameter space).
struct DevParams {
  int nx, ny, n;        // lattice, node count
  int pitch, xoff, yoff;  // padded lattice: node (x, y) at (x + xoff) + (y + yoff) * pitch
  long long plane;      // elements of one padded plane (>= pitch * (ny + 2 yoff))
  int ns;
  int periodic_x, periodic_y;
  int n_solid_list, n_wall_list;  // solid-list length, number of wall nodes
  int n_gas;            // gas-node list length
  int n_blocks;         // blocks of the fused step kernel
  int block_threads;    // its block size (the gas-tile entry cap)
  int energy_correction, coupling;
  int fixedT_face[6];   // x-, x+, y-, y+, z-, z+
  // species
  float M[MAX_NS], invM[MAX_NS], sqrtM[MAX_NS], c[MAX_NS], c2[MAX_NS];
  // sqrtM + sqrtM_lo is the reciprocal of the stored c to ~1e-14: velocities enter the
  // equilibria as v (sqrtM + sqrtM_lo), so that the equilibrium's momentum, measured with
  // c, is rho v without the constant bias c sqrtM - 1 (~1e-8) that would otherwise scale
  // the momentum at every collision.
  float sqrtM_lo[MAX_NS];
  float a[MAX_NS];      // 1 - c_j
  float ha[MAX_NS], ha2[MAX_NS];  // (1 - c_j) / 2 and (1 - c_j)^2 / 2 (interpolation)
  int onlattice[MAX_NS];
  float rref[MAX_NS];   // reference density X_inlet,j M_j of the stored deviations
  float omega[MAX_NS], t1t2[MAX_NS], wt1[MAX_NS], a2[MAX_NS], inv1a2[MAX_NS];
  float uc_w[MAX_NS], invtau2[MAX_NS];
  float kcoef[MAX_NS];  // energy-correction flux coefficient K_j / (C_j T)
  float W0[Q];          // rest-equilibrium weights at T_ref
  int storage;          // FDLBM_STORAGE_*: population storage type
  float hs[MAX_NS], hsi[MAX_NS];  // FP16 storage: power-of-two scale per species and inverse (else 1)
  float Tref, p_out;    // lattice reference temperature, outlet pressure
  float u_inlet;
  // solid and coupling
  float alpha_s, rhocp_s, inv_rhocp_s, kappa_f, dTout;
  // reactions
  int nr;
  int nu[MAX_NR][MAX_NS];
  int rate_form[MAX_NR];
  float k0[MAX_NR], EaR[MAX_NR], inv_Keq[MAX_NR], heat[MAX_NR];  // heat = -dH / (3 R T0)
  float T3T0;           // kelvin per lattice temperature unit
  float rho_w_tol;
  int rho_w_maxit;
  // steady-state residual references
  float Xin[MAX_NS];
  float Tin_lat;
  float Tdev_off;       // T_ref - T_inlet (lattice): T_ref is T_inlet rounded to a multiple of 2^-12
  // D3Q19 lattice (dim 3): node (x, y, z) at (x + xoff) + (y + yoff) pitch + (z + zoff) slab
  int dim;              // 2 (D2Q9) or 3 (D3Q19)
  int nz, zoff, periodic_z;
  long long slab;       // padded cells of one z layer
  float W0_19[19];      // D3Q19 rest-equilibrium weights at T_ref
  // locally updated relaxation times
  int local_tau;
  float mu_l[MAX_NS];               // species viscosities
  float phi_w[MAX_NS][MAX_NS];      // Wilke coefficients phi_jk
  float invD[MAX_NS][MAX_NS];       // 1 / D_jk (0 on the diagonal)
  float kcoef0[MAX_NS];             // energy-correction flux coefficient per unit tau1
  // exact accounts: the step also measures face fluxes and scheme defects (FP32 D2Q9)
  int ledger_detail;
};

// Device state of one handle.
struct DevState {
  void* h[2];           // populations (deviations from rref W0), [ns][Q][plane] padded, of the
                        // storage type (float, __nv_bfloat16 or __half)
  float* Ts[2];         // solid temperature deviation from Tref, [n]
  uint32_t* code;       // node code words on the padded lattice, [plane]
  int32_t* solid_list;  // wall nodes first, then interior solid nodes (compact indices)
  int2* gas_list;       // gas nodes {padded index, aux} (aux: GAS_AUX_*); D2Q9: per tile, its
                        // interior row-major, then its halo
  float* F[2];          // D3Q19: moment field [1 + ns][plane] of the current step: dTg, K_j
  int4* blocks;         // step-kernel block descriptors: gas tiles {0, first, interior << 16 | total,
                        // map row stride}, solid blocks {1, first, count, 0}
  uint16_t* gas_slot;   // D2Q9: moment-map slot of every gas-list entry within its tile
  float* mom;           // moments of the last step: rho_j [ns], ux, uy, T(lattice) per node, [(ns+3)][n]
  float* Tgas;          // gas temperature (lattice) for the paper coupling, [2][n] ping-pong with h
  float* snap;          // residual snapshot [(ns + 4)][n]
  double* ledger;       // FP64 ledger accumulators, LG_COUNT per solid-kernel block
  int* flags;           // sticky error flags
  float* rw;            // converged wall densities of the last step, [ns][n_wall_list] (NaN: none)
  double* red;          // reduction scratch (doubles)
  uint64_t* code64;     // D3Q19: node code words on the padded lattice, [plane]
  float2* wall_u;       // velocity of each wall-list entry (moving walls), or nullptr
};

// FP64 ledger increments per step-kernel block. The first five are always kept; the rest
// only by the exact-accounts step (ledger_detail): shift-sense energy fluxes through the
// inlet and outlet faces, the interpolation defect (pulled minus pure-shift values, gas
// pulls and wall arrivals), the collision's energy change, the wall exchange measured
// from the stored emissions and the pulled arrivals, and the solid's enthalpy change
// measured from the stored temperatures.
enum Ledger {
  LG_QRXN = 0, LG_QWALL, LG_QCOUPLE, LG_QFIXEDT, LG_NOCONV,
  LG_QIN, LG_QOUT, LG_DINT, LG_DCOL, LG_QWALLX, LG_DH, LG_COUNT
};

// Launchers (fdlbm_kernels.cu).
// Initial state from device FP64 fields: X [ns][n], u [2][n], T_lat [n], Ts_lat [n], C [n];
// inlet holds the ny inlet velocities, then the ns inlet mole fractions, then the inlet
// lattice temperature.
cudaError_t launch_init(const DevParams& P, const DevState& S, const double* X, const double* u,
                        const double* T_lat, const double* Ts_lat, const double* C,
                        const double* inlet, cudaStream_t st);
// One time step reading buffer src and writing 1 - src (step: the step's index, which
// seeds the stochastic rounding of 16-bit population storage); with moments_only the gas
// kernel recomputes the pre-collision moments of the step that read src into S.mom
// instead.
cudaError_t launch_step(const DevParams& P, const DevState& S, int src, bool moments_only,
                        cudaStream_t st, uint32_t step = 0);
// Step-kernel block size: one gas, wall or solid node per thread.
constexpr int STEP_BLOCK = 256;
// Moment-map slots of one D2Q9 gas tile: the host keeps (columns + 2)(rows + 2) within it.
constexpr int GAS_MAP_SLOTS = 640;
// Second word of a gas-list entry: the compact lattice index n = x + nx y in the low 29
// bits; GAS_AUX_GHOST marks a node (or its outlet neighbour) within GHOST of a periodic
// face, which also writes ghost copies; GAS_AUX_OUTLET a node whose +x neighbour is an
// outlet node.
constexpr int GAS_AUX_N = (1 << 29) - 1;
constexpr int GAS_AUX_OUTLET = 1 << 29;
constexpr int GAS_AUX_GHOST = 1 << 30;
// Per-block ledger slots of the step kernel and their sum (LG_COUNT doubles into out).
int ledger_slots(const DevParams& P);
cudaError_t launch_ledger_sum(const DevParams& P, const DevState& S, double* out, cudaStream_t st);
// Moment fields (FDLBM_MOMENTS layout); t_dev: T and T_s as deviations from T_inlet (K).
cudaError_t launch_moments_out(const DevParams& P, const DevState& S, int cur, float* dst, bool t_dev,
                               cudaStream_t st);
cudaError_t launch_populations_out(const DevParams& P, const DevState& S, int cur, float* dst,
                                   cudaStream_t st);
cudaError_t launch_totals(const DevParams& P, const DevState& S, int cur, cudaStream_t st);
cudaError_t launch_residual(const DevParams& P, const DevState& S, int cur, cudaStream_t st);

// Batched stepping of several handles' lattices in one launch per step.
struct BatchLaunch {
  const DevParams* params;  // [members] device parameters
  const DevState* states;   // [members] device buffers
  const int2* members;      // [members] {buffer of time level t at counter 0, step index at counter 0}
  const int4* blocks;       // {2 member + role, first, count, member-local block}
  uint32_t* counter;        // steps taken since members[] was written
  int n_blocks, ns, energy_correction, storage;
};
// One batched step (the step kernel, then the counter advance) on stream st.
cudaError_t launch_batch_step(const BatchLaunch& B, cudaStream_t st);

// ---- D3Q19 lattice (fdlbm3d_kernels.cu) ----------------------------------------------
constexpr int Q19 = 19;
// Ghost layers of the padded 3D lattice (the deepest pull reaches 3 nodes upstream).
constexpr int GHOST3 = 3;
constexpr int XOFF3 = 4;
// 64-bit code word of a 3D node: class (bits 0..2), catalytic (3), 3-bit streaming
// stencil per direction i = 1..18 at bit 4 + 3 (i - 1), and at bit 58 + (d - 1) for the
// axis directions d = 1..6 a gas neighbour (gas nodes) or a solid neighbour (solid
// nodes).
constexpr int STENCIL_SHIFT3 = 4;
constexpr int NBR_SHIFT3 = 58;
__host__ __device__ inline uint32_t node_class3(uint64_t code) { return uint32_t(code & 7u); }
__host__ __device__ inline uint32_t stencil_of3(uint64_t code, int i) {
  return uint32_t(code >> (STENCIL_SHIFT3 + 3 * (i - 1))) & 7u;
}
// Step-kernel block size of the 3D path.
constexpr int STEP_BLOCK3 = 128;
// Doubles written by the 3D totals / residual reductions.
inline int residual_count3(int ns) { return 2 * (ns + 5); }
cudaError_t launch_init3(const DevParams& P, const DevState& S, const double* X, const double* u,
                         const double* T_lat, const double* Ts_lat, const double* C, const double* inlet,
                         cudaStream_t st);
// One 3D time step reading buffer src (step: the step's index, which seeds the stochastic
// rounding of 16-bit storage); with moments_only the pre-collision moments into S.mom.
cudaError_t launch_step3(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st,
                         uint32_t step = 0);
cudaError_t launch_moments_out3(const DevParams& P, const DevState& S, int cur, float* dst, bool t_dev,
                                cudaStream_t st);
cudaError_t launch_populations_out3(const DevParams& P, const DevState& S, int cur, float* dst,
                                    cudaStream_t st);
cudaError_t launch_totals3(const DevParams& P, const DevState& S, int cur, cudaStream_t st);
cudaError_t launch_residual3(const DevParams& P, const DevState& S, int cur, cudaStream_t st);

// One D2Q9 step with locally updated relaxation times (FP32 storage; fdlbm_local_tau.cu);
// with moments_only the pre-collision moments of the step that reads src into S.mom.
cudaError_t launch_step_local_tau(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st,
                                  uint32_t step);
// One D2Q9 step that also keeps the exact accounts (FP32 storage; fdlbm_ledger_detail.cu).
cudaError_t launch_step_detail(const DevParams& P, const DevState& S, int src, cudaStream_t st, uint32_t step);
// Energy sum (1/2) c_j^2 |e_i|^2 g of the stored populations of gas nodes and of the wall
// emissions in transit (FP32 storage), added into *out (zeroed here first).
cudaError_t launch_pop_energy(const DevParams& P, const DevState& S, int cur, double* out, cudaStream_t st);

// Bytes of one stored population.
inline size_t pop_bytes_per_value(int storage) { return storage == FDLBM_STORAGE_FP32 ? 4 : 2; }

// Number of doubles written by launch_totals into S.red: E_gas, H_solid, mass[ns], moles[ns].
inline int totals_count(int ns) { return 2 + 2 * ns; }
// Number of doubles written by launch_residual into S.red (after the totals):
// per field: ||F - snap||^2 and ||F - ref||^2 for fields ux, uy, X_j, T, Ts.
inline int residual_count(int ns) { return 2 * (ns + 4); }

// Allocation-free totals: the same sums as launch_totals, reduced in a fixed order
// through the library's static device scratch of FDLBM_STATIC_SCRATCH_BYTES.
constexpr int TOTALS_STATIC_BLOCK = 256;
// Doubles of scratch the reduction needs: one partial row per block plus the totals.
inline long long totals_static_doubles(long long n_nodes, int ns) {
  return ((n_nodes + TOTALS_STATIC_BLOCK - 1) / TOTALS_STATIC_BLOCK + 1) * totals_count(ns);
}
// Device address of the static scratch on the current device (cudaGetSymbolAddress).
cudaError_t totals_static_scratch(double** out);
// Partial sums into scratch[0, blocks * count), totals into the next count doubles.
cudaError_t launch_totals_static(const DevParams& P, const DevState& S, int cur, double* scratch,
                                 cudaStream_t st);

}  // namespace fdlbm
