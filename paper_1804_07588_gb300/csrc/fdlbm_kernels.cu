// CUDA kernels of the coupled FD-LBM solver (sm_103a).
//
// Storage. Populations are FP32 deviations h = g - rref_j W0_i from the rest equilibrium
// of the inlet state (rref_j = X_inlet,j M_j, W0 = f^eq(1, 0, T_ref)); the solid
// temperature is stored as T_s - T_ref. Every moment and equilibrium is evaluated in that
// deviation form, so FP32 keeps the precision the FP64 reference needs. Population planes
// [species][direction] live on a padded lattice with GHOST = 4 ghost layers around the
// nodes: a node within GHOST of a periodic face also writes its populations into the
// ghost copy on the other side, so every pull is a plain linear offset.
//
// One time step is one launch of step_kernel, whose blocks take a gas or a solid role
// (both read time level t only):
//   solid role: interface (wall) nodes stream in the populations arriving from the gas,
//     iterate the wall density with the surface reaction (Sec. 4.3, Eq. BC_gji), emit the
//     unknown populations and apply the FD heat step with the interface coupling and the
//     reaction heat (Sec. 5); interior solid nodes apply the FD step only.
//   gas role: one thread per entry of a compact list of gas nodes: fused pull streaming
//     with the off-lattice interpolation (Sec. 4.2) into thread-private shared memory,
//     moments (Eq. moments_of_g), divergence of the energy-correction flux from the
//     moment field of the previous time level, two-step collision (Eq.
//     final_kinetic_equation), outlet equilibrium; it writes this step's moment field.
#include "fdlbm_device.cuh"

namespace fdlbm {

// The 16-bit storage paths are instantiated in their own translation units.
FDLBM_STORAGE_ENTRY_POINTS(extern, __nv_bfloat16)
FDLBM_STORAGE_ENTRY_POINTS(extern, __half)
FDLBM_STORAGE_ENTRY_POINTS(, float)

namespace {

// Sum of the per-block ledger slots.
__global__ void ledger_sum_kernel(const double* __restrict__ slots, int nblocks, double* __restrict__ out) {
  const int t = threadIdx.x;
  if (t >= LG_COUNT) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += slots[(long long)b * LG_COUNT + t];
  out[t] = s;
}

__global__ void zero_solid_ts(DevParams P, float* __restrict__ Ts0, float* __restrict__ Ts1) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < P.n) Ts0[n] = Ts1[n] = 0.f;
}

// ---------------------------------------------------------------------------------------
// Outputs and reductions (compact node indices)
// ---------------------------------------------------------------------------------------
// T and T_s in kelvin, or with dev as deviations from the inlet temperature (kelvin).
__global__ void moments_out_kernel(DevParams P, const float* __restrict__ mom, const float* __restrict__ Ts,
                                   const uint32_t* __restrict__ code, float* __restrict__ dst, int dev) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P.n) return;
  const int ns = P.ns;
  const uint32_t c = node_class(code[pad_index(P, n % P.nx, n / P.nx)]);
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
    dst[(2 * ns + 2) * N + n] = (dev ? mom[(ns + 2) * N + n] + P.Tdev_off : P.Tref + mom[(ns + 2) * N + n]) * P.T3T0;
  } else if (c == WALL || c == SOLID) {
    dst[(2 * ns + 3) * N + n] = (dev ? Ts[n] + P.Tdev_off : P.Tref + Ts[n]) * P.T3T0;
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
  for (int f = 0; f < nf; ++f) cur[f] = 0.f;
  if (n < P.n) {
    const uint32_t c = node_class(code[pad_index(P, n % P.nx, n / P.nx)]);
    on_gas = c == GAS;
    on_solid = c == WALL || c == SOLID;
    if (on_gas) {
      float C = 0.f;
      for (int j = 0; j < ns; ++j) C += mom[j * N + n] * P.invM[j];
      cur[0] = mom[ns * N + n];
      cur[1] = mom[(ns + 1) * N + n];
      for (int j = 0; j < ns; ++j) cur[2 + j] = mom[j * N + n] * P.invM[j] / C;
      cur[2 + ns] = mom[(ns + 2) * N + n];  // T - T_ref
    }
    if (on_solid) cur[3 + ns] = Ts[n];
  }
  for (int f = 0; f < nf; ++f) {
    const bool on = f == nf - 1 ? on_solid : on_gas;
    double dd = 0.0, dr = 0.0;
    if (on) {
      const double ref = f < 2 ? 0.0 : (f < 2 + ns ? double(P.Xin[f - 2]) : -double(P.Tdev_off));
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

static_assert(2 + 2 * MAX_NS <= 64, "one thread per totals column in a 64-thread block");

// Column q of the partial rows summed in block order into out[q] (one thread per column).
__global__ void totals_rows_kernel(const double* __restrict__ part, int rows, int cnt,
                                   double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q >= cnt) return;
  double s = 0.0;
  for (int b = 0; b < rows; ++b) s += part[(long long)b * cnt + q];
  out[q] = s;
}

}  // namespace

cudaError_t launch_init(const DevParams& P, const DevState& S, const double* X, const double* u,
                        const double* T_lat, const double* Ts_lat, const double* C, const double* inlet,
                        cudaStream_t st) {
  zero_solid_ts<<<(P.n + 255) / 256, 256, 0, st>>>(P, S.Ts[0], S.Ts[1]);
  switch (P.storage) {
    case FDLBM_STORAGE_FP32: return storage_init<float>(P, S, X, u, T_lat, Ts_lat, C, inlet, st);
    case FDLBM_STORAGE_BF16: return storage_init<__nv_bfloat16>(P, S, X, u, T_lat, Ts_lat, C, inlet, st);
    case FDLBM_STORAGE_FP16: return storage_init<__half>(P, S, X, u, T_lat, Ts_lat, C, inlet, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st,
                        uint32_t step) {
  switch (P.storage) {
    case FDLBM_STORAGE_FP32: return storage_step<float>(P, S, src, moments_only, st, step);
    case FDLBM_STORAGE_BF16: return storage_step<__nv_bfloat16>(P, S, src, moments_only, st, step);
    case FDLBM_STORAGE_FP16: return storage_step<__half>(P, S, src, moments_only, st, step);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_step(const BatchLaunch& B, cudaStream_t st) {
  switch (B.storage) {
    case FDLBM_STORAGE_FP32: return storage_batch_step<float>(B, st);
    case FDLBM_STORAGE_BF16: return storage_batch_step<__nv_bfloat16>(B, st);
    case FDLBM_STORAGE_FP16: return storage_batch_step<__half>(B, st);
    default: return cudaErrorInvalidValue;
  }
}

int ledger_slots(const DevParams& P) { return P.n_blocks > 0 ? P.n_blocks : 1; }

cudaError_t launch_ledger_sum(const DevParams& P, const DevState& S, double* out, cudaStream_t st) {
  ledger_sum_kernel<<<1, 32, 0, st>>>(S.ledger, ledger_slots(P), out);
  return cudaGetLastError();
}

cudaError_t launch_moments_out(const DevParams& P, const DevState& S, int cur, float* dst, bool t_dev,
                               cudaStream_t st) {
  const int nb = (P.n + 255) / 256;
  moments_out_kernel<<<nb, 256, 0, st>>>(P, S.mom, S.Ts[cur], S.code, dst, t_dev ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_populations_out(const DevParams& P, const DevState& S, int cur, float* dst, cudaStream_t st) {
  switch (P.storage) {
    case FDLBM_STORAGE_FP32: return storage_populations_out<float>(P, S, cur, dst, st);
    case FDLBM_STORAGE_BF16: return storage_populations_out<__nv_bfloat16>(P, S, cur, dst, st);
    case FDLBM_STORAGE_FP16: return storage_populations_out<__half>(P, S, cur, dst, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_totals(const DevParams& P, const DevState& S, int cur, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(S.red, 0, sizeof(double) * totals_count(P.ns), st);
  if (e != cudaSuccess) return e;
  switch (P.storage) {
    case FDLBM_STORAGE_FP32: return storage_totals<float>(P, S, cur, st);
    case FDLBM_STORAGE_BF16: return storage_totals<__nv_bfloat16>(P, S, cur, st);
    case FDLBM_STORAGE_FP16: return storage_totals<__half>(P, S, cur, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_residual(const DevParams& P, const DevState& S, int cur, cudaStream_t st) {
  double* out = S.red + totals_count(P.ns);
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * residual_count(P.ns), st);
  if (e != cudaSuccess) return e;
  const int nb = (P.n + 255) / 256;
  residual_kernel<<<nb, 256, 0, st>>>(P, S.mom, S.Ts[cur], S.code, S.snap, out);
  return cudaGetLastError();
}

// The scratch itself: FDLBM_STATIC_SCRATCH_BYTES reserved with the library's device
// code, one copy per device. Reached only through totals_static_scratch.
static __device__ __align__(256) double g_totals_static[FDLBM_STATIC_SCRATCH_BYTES / sizeof(double)];

cudaError_t totals_static_scratch(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_totals_static);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

cudaError_t launch_totals_static(const DevParams& P, const DevState& S, int cur, double* scratch,
                                 cudaStream_t st) {
  const int cnt = totals_count(P.ns);
  const int nb = (P.n + TOTALS_STATIC_BLOCK - 1) / TOTALS_STATIC_BLOCK;
  if (totals_static_doubles(P.n, P.ns) * (long long)sizeof(double) > FDLBM_STATIC_SCRATCH_BYTES)
    return cudaErrorInvalidValue;
  if (nb > 0) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (P.storage) {
      case FDLBM_STORAGE_FP32: e = storage_totals_partial<float>(P, S, cur, scratch, nb, st); break;
      case FDLBM_STORAGE_BF16: e = storage_totals_partial<__nv_bfloat16>(P, S, cur, scratch, nb, st); break;
      case FDLBM_STORAGE_FP16: e = storage_totals_partial<__half>(P, S, cur, scratch, nb, st); break;
      default: break;
    }
    if (e != cudaSuccess) return e;
  }
  totals_rows_kernel<<<1, 64, 0, st>>>(scratch, nb, cnt, scratch + (long long)nb * cnt);
  return cudaGetLastError();
}

}  // namespace fdlbm
