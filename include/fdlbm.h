/* fdlbm.h — C ABI of the GB300 (sm_103a) solver for the coupled finite-difference /
 * lattice-Boltzmann scheme for catalytic flow of Kulyk, Berger, Smith and Harting,
 * "Catalytic flow with a coupled Finite Difference - Lattice Boltzmann scheme"
 * (arXiv:1804.07588).
 *
 * One time step of the solver is the paper's scheme on a D2Q9 lattice:
 *   - the multicomponent thermal LBM gas (Sec. 2-4): one population set per species,
 *     off-lattice quadratic interpolation while streaming heavy species (Sec. 4.2),
 *     two-step quasi-equilibrium collision of the transformed populations g with the
 *     diffusion-velocity and energy correction terms (Eq. final_kinetic_equation);
 *   - reactive diffusive-wall boundary conditions on gas-solid interface nodes with the
 *     iterated wall density (Sec. 4.3, Eq. BC_gji);
 *   - the explicit FD heat equation in the solid coupled through the interface nodes,
 *     which also receive the reaction heat (Sec. 5, Eqs. heat_equation_fd,
 *     wall_temperature).
 *
 * Conventions (every call):
 *   - Every function returns an fdlbm_status; nothing throws across the ABI.
 *   - Host pointers passed to fdlbm_create / fdlbm_set_fields are read during the call
 *     only (the library copies what it needs); the caller keeps ownership.
 *   - Output buffers are caller-owned. Device output pointers must be device memory of
 *     the handle's device; transfers and kernels run on the handle's stream.
 *   - Device memory is taken from the caller's allocator (fdlbm_options.alloc) or
 *     cudaMalloc and released by fdlbm_destroy.
 *   - Lattice nodes are indexed n = x + nx * y (2D) or n = x + nx * (y + ny * z) (3D),
 *     x fastest; field arrays are [field][n] in that order.
 *   - D3Q19 handles (fdlbm_geometry.lattice = FDLBM_D3Q19) support create, step, sync,
 *     moments, populations, enthalpy balance, residual, set_fields, info, profiling and
 *     destroy with any population storage and a plug inlet; checkpoints, batches and
 *     the allocation-free totals are D2Q9 only and return EINVAL for a 3D handle.
 *   - Error messages of the last failing call on this thread: fdlbm_last_error().
 */
#ifndef FDLBM_H
#define FDLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDLBM_MAX_SPECIES 6
#define FDLBM_MAX_REACTIONS 4

typedef struct fdlbm_handle fdlbm_handle; /* opaque, library-owned */

typedef enum {
  FDLBM_OK = 0,
  FDLBM_EINVAL = -1,    /* bad argument or unsupported combination */
  FDLBM_EGEOM = -2,     /* geometry rejected (gas touching a closed face, bad outlet) */
  FDLBM_ECUDA = -3,     /* CUDA runtime error */
  FDLBM_EUNSTABLE = -4, /* the gas kernel saw a non-finite or non-positive density/temperature */
  FDLBM_ENOCONV = -5,   /* reserved: wall-density iteration cap reached (counted, see balance) */
  FDLBM_ETIMEOUT = -6,  /* reserved for bounded device waits */
  FDLBM_ENOMEM = -7,    /* device allocation failed */
  FDLBM_EIO = -8        /* checkpoint file missing, unreadable, truncated or not written */
} fdlbm_status;

/* Lattices: the paper's D2Q9 and the D3Q19 extension it announces (Sec. 2), built from
 * the D3Q27 product-form equilibrium by folding each corner population onto its three
 * face diagonals (+), its three axis links (-) and the rest population (+). */
enum { FDLBM_D2Q9 = 9, FDLBM_D3Q19 = 19 };
/* Face boundary kinds for faces x-, x+, y-, y+ (indices 0..3). Periodic faces come in
 * pairs; inlet only on x-, outlet only on x+. */
enum { FDLBM_FACE_PERIODIC = 0, FDLBM_FACE_INLET = 1, FDLBM_FACE_OUTLET = 2,
       FDLBM_FACE_CLOSED = 3, FDLBM_FACE_FIXED_T = 4 };
/* Geometry mask values. */
enum { FDLBM_MASK_GAS = 0, FDLBM_MASK_INERT = 1, FDLBM_MASK_CATALYTIC = 2 };
enum { FDLBM_PROFILE_PLUG = 0, FDLBM_PROFILE_PARABOLIC = 1 };
/* Interface coupling: CONSERVATIVE gives the solid exactly the energy its diffusive
 * wall took from the gas; PAPER is the wall-temperature law of Eq. wall_temperature. */
enum { FDLBM_COUPLING_CONSERVATIVE = 0, FDLBM_COUPLING_PAPER = 1 };
/* Surface rate laws: k C_a C_b of Eq. showcase_Sj, or the reversible mole-fraction
 * law k (prod x_reactants - prod x_products / Keq). */
enum { FDLBM_RATE_CONC_BILINEAR = 0, FDLBM_RATE_XFRAC_REVERSIBLE = 1 };
/* Population storage. Every population is stored as its deviation from the rest
 * equilibrium of the inlet state, g - rho_ref,j w_i(T_ref); the arithmetic is FP32 for
 * every storage type. BF16 rounds each stored deviation to 8 significant bits; FP16 to
 * 11, after scaling it by a power of two per species chosen from the species' molar
 * mass so that deviations up to twice its molar mass stay in FP16's range. */
enum { FDLBM_STORAGE_FP32 = 0, FDLBM_STORAGE_BF16 = 1, FDLBM_STORAGE_FP16 = 2 };

/* Lattice and geometry (Sec. 4.3: walls sit on the solid nodes next to the gas). */
typedef struct {
  int nx, ny;              /* lattice size, each >= 4 */
  int lattice;             /* FDLBM_D2Q9 or FDLBM_D3Q19 */
  const uint8_t* mask;     /* host, nx*ny (2D) or nx*ny*nz (3D), x fastest then y, FDLBM_MASK_* */
  int face_bc[6];          /* FDLBM_FACE_* for x-, x+, y-, y+, z-, z+ (z faces: 3D only); a
                              periodic axis needs at least 8 nodes (D2Q9) or 6 (D3Q19) */
  int nz;                  /* D3Q19: z size >= 4; ignored for D2Q9 */
  /* Optional (D2Q9, may be NULL): host [2][n] lattice velocity of solid nodes. An
   * interface wall node with a velocity U_w is a moving diffusive wall: it emits
   * f^eq_j(1, U_w, T_w) (Eq. BC_g_ji_1 with the wall velocity) in place of the rest
   * weights. The solid's FD heat step is unchanged; with FDLBM_COUPLING_CONSERVATIVE the
   * mechanical work the wall does on the gas is charged to the solid's enthalpy. */
  const double* wall_u;
} fdlbm_geometry;

/* One gas species (Sec. 2; relaxation times in lattice units). */
typedef struct {
  double M_gmol;           /* molar mass; the lightest species streams on-lattice */
  double tau1, tau2;       /* relaxation times of Eq. bare_kinetic_eq, > 0 (constant mode) */
  double X_init, X_inlet;  /* default initial and inlet mole fractions */
  /* Locally updated relaxation times (fdlbm_transport.local_tau = 1, Sec. 3): the
   * species viscosity (lattice units) and the binary diffusivities D[k] with every other
   * species k (lattice units, > 0; D[j] of the species itself is unused). */
  double mu;
  double D[FDLBM_MAX_SPECIES];
} fdlbm_species;

/* Transport, thermal and solid parameters. Temperatures in kelvin; the lattice
 * temperature is T / (3 T0) (Sec. 4.1). */
typedef struct {
  double Pr;               /* Prandtl number of the energy correction (Eq. q_Pr) */
  int energy_correction;   /* 1: apply the energy correction Phi, 0: none */
  double T0_K, T_init_K, T_inlet_K, T_solid_init_K, T_outer_K;
  double u_inlet;          /* inlet velocity (peak for the parabolic profile), lattice */
  int inlet_profile;       /* FDLBM_PROFILE_* */
  double alpha_s;          /* solid thermal diffusivity, lattice (Eq. heat_equation_fd) */
  double rhocp_s;          /* solid volumetric heat capacity, lattice energy / lattice T */
  double kappa_f;          /* gas conductivity used by FDLBM_COUPLING_PAPER */
  int coupling;            /* FDLBM_COUPLING_* */
  /* 1: relaxation times updated at every gas node and step from the local composition
   * and temperature (Sec. 3): tau1_j = mu_j / (C T sum_k X_k phi_jk) with Wilke's phi_jk
   * (Eqs. wilke, tau1s; the bracket of phi_jk squared, as in Wilke's rule) and
   * tau2_j = rho_j D_j / (X_j p), D_j = (1 - Y_j) / sum_{k != j} X_k / D_jk (Eqs.
   * tau2_approx_text, D_j_text), from the pulled densities and the g-temperature of
   * the step. D2Q9 with FP32 storage and at least 2 species; not in batches. */
  int local_tau;
} fdlbm_transport;

/* Surface reactions on catalytic wall nodes (Sec. 4.3 and Sec. 6). */
typedef struct {
  int n_react;
  int nu[FDLBM_MAX_REACTIONS][FDLBM_MAX_SPECIES]; /* stoichiometry, <0 reactants */
  double k0[FDLBM_MAX_REACTIONS];      /* lattice moles per wall node per step */
  double Ea_Jmol[FDLBM_MAX_REACTIONS];
  double Keq[FDLBM_MAX_REACTIONS];
  double dH_Jmol[FDLBM_MAX_REACTIONS]; /* reaction enthalpy, < 0 exothermic */
  int rate_form[FDLBM_MAX_REACTIONS];  /* FDLBM_RATE_* */
  double rho_w_tol;                    /* wall-density iteration tolerance (1e-8) */
  int rho_w_maxit;                     /* iteration cap */
} fdlbm_kinetics;

/* Optional initial fields (host, may be NULL individually): mole fractions [ns][n],
 * velocity [D][n] (lattice, D = 2 or 3), gas and solid temperatures [n] (K), molar
 * concentration [n] (lattice, default 1). */
typedef struct {
  const double* X;
  const double* u;
  const double* T_K;
  const double* Ts_K;
  const double* C;
} fdlbm_fields;

/* Device memory and stream. alloc/free may be NULL (cudaMalloc / cudaFree). stream is a
 * cudaStream_t (NULL: the legacy default stream). */
typedef struct {
  int storage;             /* FDLBM_STORAGE_* (FP32 default) */
  int device;              /* CUDA device ordinal */
  void* stream;
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* ctx);
  void* alloc_ctx;
  int band_rows;           /* D2Q9: rows per band of the step kernel's block order (the gas
                              tiles of a band, then its wall blocks) and height of the gas
                              tiles, at most 64; 0: 16 */
  int ledger_detail;       /* 1: every step also keeps the exact accounts of fdlbm_balance
                              (E_pop ... closure); FP32 storage and constant relaxation
                              times only (else EINVAL); slower steps, same results */
  int strict_geometry;     /* 1: reject (EGEOM, naming the first such node) geometries whose
                              pulls need the linear or no-interpolation fallbacks, i.e.
                              concave corners and one- or two-node gaps; the paper
                              restricts its walls to planar and convex corner nodes
                              (Sec. 4.2, Sec. 4.3). 0: accept them, with the fallbacks */
  int tile_entries;        /* D2Q9: at most this many gas nodes (interior and halo ring) per
                              gas tile, which is also the step kernel's block size: a
                              multiple of 32 in [64, 256]; 0: 256. EINVAL otherwise */
  int wall_order;          /* D2Q9 block order: 0 each band's wall and solid blocks right
                              after its gas tiles (their neighbours' populations still in
                              L2); 1 all wall and solid blocks after all gas tiles */
} fdlbm_options;

/* Counts and derived constants of a handle. */
typedef struct {
  int64_t n_nodes, n_gas, n_inlet, n_outlet, n_wall, n_solid;
  int64_t stencil_counts[6]; /* gas + wall pull directions by stencil: none, central,
                                forward, backward, linear-s0, linear-s2 */
  int ns;
  double T_ref_lat;          /* lattice reference temperature T_inlet / (3 T0) */
  int64_t steps;
  size_t device_bytes;       /* device memory held by the handle */
} fdlbm_info_t;

/* FP64 ledger (Sec. 5, enthalpy conservation; lattice energy units, energy of the gas
 * = internal + kinetic from the f-moments plus the populations emitted by walls and not
 * yet streamed into the gas). */
typedef struct {
  int64_t steps;
  double E_gas, E_gas0, H_solid, H_solid0;
  double Q_reaction;       /* cumulative reaction heat released into wall nodes */
  double Q_wall;           /* cumulative energy the diffusive walls put into the gas */
  double Q_couple;         /* cumulative energy the solid received from the gas coupling */
  double Q_fixedT;         /* cumulative heat into the solid through fixed-T faces */
  double residual;         /* dE_gas + dH_solid - Q_reaction - Q_fixedT */
  double solid_residual;   /* dH_solid - (Q_reaction + Q_couple + Q_fixedT) */
  double eps_paper;        /* Eq. error_coupling with the gas-phase change of the first
                              reactant of reaction 0 */
  double noconv;           /* wall-density iterations that hit the cap */
  double mass[FDLBM_MAX_SPECIES], mass0[FDLBM_MAX_SPECIES];
  double moles[FDLBM_MAX_SPECIES], moles0[FDLBM_MAX_SPECIES];
  /* Exact accounts (handles created with ledger_detail; otherwise zero, closure NaN).
   * Inventory: energy (1/2) c_j^2 |e_i|^2 g of the stored populations of gas nodes and
   * of the wall emissions in transit. Per step, FP64 sums of exact differences of the
   * FP32 values stored and pulled:
   *   Q_inlet, Q_outlet: energy gas nodes pull from inlet / outlet nodes as their shift
   *     source (s1) minus the energy of their populations that stream into them;
   *   D_interp: departure of each interpolated pull from the pure shift (Sec. 4.2), at
   *     gas nodes and wall arrivals (zero for species with c_j = 1);
   *   D_collision: energy change of the collision (Eq. final_kinetic_equation);
   *   D_coupling: energy the walls put into the gas (stored emissions minus pulled
   *     arrivals) plus Q_couple: zero up to the FP32 rounding of the exchange the solid
   *     receives in the conservative coupling, the imbalance of Eq. wall_temperature in
   *     the paper's;
   *   D_solid: change of H_solid from the stored temperatures minus Q_reaction +
   *     Q_couple + Q_fixedT (the FP32 rounding of the FD step).
   * closure = (E_pop - E_pop0) + (H_solid - H_solid0) - Q_reaction - Q_fixedT - Q_inlet -
   *   Q_outlet - D_interp - D_collision - D_coupling - D_solid: FP64 rounding. */
  double E_pop, E_pop0;
  double Q_inlet, Q_outlet, D_interp, D_collision, D_coupling, D_solid;
  double closure;
  int ledger_detail;
} fdlbm_balance;

/* Build a solver: validate, convert units, classify nodes (gas / inlet / outlet /
 * interface wall / solid), precompute the streaming stencil of every pull, allocate
 * device state and initialise g* = f^eq(initial fields), wall emissions and T_s.
 * init and opts may be NULL. On success *out owns device memory until fdlbm_destroy.
 * Errors: EINVAL (parameters), EGEOM (geometry), ENOMEM, ECUDA. */
fdlbm_status fdlbm_create(const fdlbm_geometry* geom, const fdlbm_species* species, int n_species,
                          const fdlbm_transport* tr, const fdlbm_kinetics* kin,
                          const fdlbm_fields* init, const fdlbm_options* opts, fdlbm_handle** out);

/* Enqueue n >= 0 time steps on the handle's stream (asynchronous). A D2Q9 step is one
 * launch of the fused step kernel: gas tiles (streaming, moments, the energy-correction
 * divergence from this step's moments, collision, Sec. 4), interface wall nodes
 * (reactive diffusive wall, Sec. 4.3) and solid nodes (FD heat step and coupling,
 * Sec. 5) in one grid. A D3Q19 step with the energy correction first writes this step's
 * moment field in a pass over the gas nodes, then launches the step kernel. */
fdlbm_status fdlbm_step(fdlbm_handle* h, int64_t n);

/* Wait for the handle's stream and report sticky device errors (EUNSTABLE). */
fdlbm_status fdlbm_sync(fdlbm_handle* h);

/* Moment fields at the current time into dst, [2 ns + 2 + D][n] float32: rho_j, X_j, ux,
 * uy (, uz), T (K) on gas nodes, T_s (K) on solid nodes, 0 elsewhere. dst_on_device
 * selects a device or host destination; a host copy is synchronous. */
fdlbm_status fdlbm_moments(fdlbm_handle* h, float* dst, int dst_on_device);

/* fdlbm_moments with flags. FDLBM_MOMENTS_T_DEVIATION writes T and T_s as deviations
 * from the inlet temperature, in K: the solver keeps temperatures as deviations from its
 * reference state, and a float32 absolute temperature (ulp 3e-5 K at 500 K) would drop
 * the digits of a small departure (a 2 K deviation carries only 5 of them). Other flag
 * bits: EINVAL. */
#define FDLBM_MOMENTS_T_DEVIATION 1u
fdlbm_status fdlbm_moments_ex(fdlbm_handle* h, unsigned flags, float* dst, int dst_on_device);

/* Stored populations g* (post-collision on gas, inlet and outlet nodes, emissions on
 * wall nodes), [ns][Q][n] float32 (Q = 9 or 19; absolute values, not deviations).
 * Direction i moves along e_i (species j by c_j e_i per step, Sec. 4.2):
 *   D2Q9:  (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1);
 *   D3Q19: (0,0,0) (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1) (1,1,0) (-1,-1,0)
 *          (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1)
 *          (0,1,-1) (0,-1,1). */
fdlbm_status fdlbm_populations(fdlbm_handle* h, float* dst, int dst_on_device);

/* FP64 ledger (synchronous). */
fdlbm_status fdlbm_enthalpy_balance(fdlbm_handle* h, fdlbm_balance* out);

/* Steady-state residual since the previous call (first call: +inf), K = steps since
 * then; synchronous. */
fdlbm_status fdlbm_residual(fdlbm_handle* h, double* out);

/* Allocation-free totals. The paper has no counterpart: this is a library facility.
 *
 * Writes the conserved totals of the current time to the host array out (out_len >=
 * 2 + 2 n_species doubles): {E_gas, H_solid, mass[ns], moles[ns]}, the same quantities
 * and units as the members of fdlbm_balance filled by fdlbm_enthalpy_balance, which
 * sums them through the handle's own scratch with atomics. This call reduces in a fixed
 * order (per-block partial sums, then one pass over the blocks), so repeated calls on
 * the same state return identical bits.
 *
 * It allocates no device memory: the partial sums live in one library-wide device
 * array of FDLBM_STATIC_SCRATCH_BYTES, reserved when the library is loaded. It is for
 * callers that must not allocate at the point of the call: a monitor that polls the
 * totals while every free byte of the device is held by resident lattices; a caller
 * that must not stall its other streams, since freeing device memory waits for the
 * whole device; and code that runs on a thread where the Python caching allocator
 * must not be entered. A call issues one moments relaunch (if the moments are stale),
 * two reduction kernels and one device-to-host copy on the handle's stream, then
 * waits for that stream.
 *
 * Limit: the lattice must satisfy (ceil(nx ny / 256) + 1)(2 + 2 ns) x 8 bytes <=
 * FDLBM_STATIC_SCRATCH_BYTES, e.g. nx ny <= 698,368 for 5 species; larger lattices are
 * rejected with EINVAL and a message giving both sizes. Nothing in the scratch has to
 * start at zero: every slot the call reads was written earlier in the same call.
 *
 * The first call on a device looks up the scratch address on that device; make that
 * first call before any stream capture on the device. The scratch is shared by all
 * handles on a device: a process-wide lock, held from the start of a call until its
 * read-back has completed, makes calls from several host threads, handles or streams
 * take it one after another (a call waits for any other in progress). Errors: EINVAL
 * (NULL arguments, out_len too small, lattice over the limit), ECUDA. */
#define FDLBM_STATIC_SCRATCH_BYTES 262144
fdlbm_status fdlbm_totals_static(fdlbm_handle* h, double* out, int out_len);

/* Batched stepping (the paper has none: a library facility). A batch advances several
 * independent handles together, one kernel launch per time step covering every member's
 * gas, wall and solid blocks, with the per-step launches captured in a CUDA graph of 16
 * steps that is replayed. Members must share the device, the species count, the storage
 * type and the energy-correction switch; lattices, geometries and all other parameters
 * may differ. A member advanced by a batch gives the same results, bit for bit, as when
 * stepped alone; the handle stays usable on its own (outputs, residual, fdlbm_step) and
 * the batch notices when a member was stepped outside it. The batch does not own its
 * members: destroy the batch before them.
 * fdlbm_batch_create: EINVAL (NULL or repeated handles, incompatible members), ECUDA.
 * fdlbm_batch_step: enqueue n >= 0 steps of every member on the batch's own stream,
 *   ordered after the work already queued on the members' streams and before any work
 *   queued on them afterwards. The batch also holds a few small device tables of its own
 *   (cudaMalloc), rewritten when members change.
 * fdlbm_batch_remove: stop advancing member h (e.g. once it reached steady state). */
typedef struct fdlbm_batch fdlbm_batch;
fdlbm_status fdlbm_batch_create(fdlbm_handle* const* handles, int n, fdlbm_batch** out);
fdlbm_status fdlbm_batch_step(fdlbm_batch* b, int64_t n);
fdlbm_status fdlbm_batch_remove(fdlbm_batch* b, fdlbm_handle* h);
int fdlbm_batch_size(const fdlbm_batch* b);
void fdlbm_batch_destroy(fdlbm_batch* b);

/* Checkpoint and restore (the paper has none: a library facility). fdlbm_save writes
 * the state the next step reads (current populations, solid temperature, moments,
 * residual snapshot, ledger, wall densities, step count) to the file at path;
 * fdlbm_load restores it into a handle created from the same geometry, species,
 * transport and kinetics (checked by a fingerprint of the node codes and device
 * parameters: EINVAL otherwise). Steps after a load give the same bits as steps after
 * the save on the saving handle. Both are synchronous; the file is host-endian.
 * Errors: EINVAL, EIO, ECUDA. */
fdlbm_status fdlbm_save(fdlbm_handle* h, const char* path);
fdlbm_status fdlbm_load(fdlbm_handle* h, const char* path);

/* Re-initialise the gas (and solid) state from fields (warm start); NULL members keep
 * the defaults of fdlbm_create. The ledger is reset. */
fdlbm_status fdlbm_set_fields(fdlbm_handle* h, const fdlbm_fields* f);

fdlbm_status fdlbm_info(const fdlbm_handle* h, fdlbm_info_t* out);

/* Kernel timing for benchmarks. With enable != 0, fdlbm_step records CUDA events on the
 * handle's stream around the step kernel of each step (one launch per step; at most
 * 65536 steps are kept). fdlbm_kernel_times waits for the stream, writes the summed
 * milliseconds {step kernel, 0} and the number of timed steps, and clears the record. */
fdlbm_status fdlbm_profile(fdlbm_handle* h, int enable);
fdlbm_status fdlbm_kernel_times(fdlbm_handle* h, double* ms_out2, int64_t* steps_out);

void fdlbm_destroy(fdlbm_handle* h);

/* Message of the last failing call on this thread (library-owned, never NULL). */
const char* fdlbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
