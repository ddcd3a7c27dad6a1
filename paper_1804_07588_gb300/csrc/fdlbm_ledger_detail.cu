// D2Q9 step kernels that also keep the exact accounts of the scheme (FP32 population
// storage), and the energy inventory of the stored populations. Each step adds, per
// block and in FP64, the energy that gas nodes take from inlet and outlet nodes minus
// what they stream into them, the departure of every interpolated pull from the pure
// shift (Sec. 4.2; gas pulls and wall arrivals), the collision's energy change, the wall
// exchange measured from the stored emissions and the pulled arrivals (Sec. 4.3) and the
// solid's enthalpy change measured from the stored temperatures (Sec. 5). Each increment
// is an exact difference of FP32 values, so the energy balance closes to FP64 rounding.
// Its own translation unit, so that the library's translation units compile in parallel.
#include "fdlbm_device.cuh"

namespace fdlbm {

namespace {
template <int NS>
cudaError_t detail_ns(const DevParams& P, const DevState& S, int src, cudaStream_t st, uint32_t step) {
  return P.energy_correction ? step_launch<float, NS, true, false, true>(P, S, src, st, step)
                             : step_launch<float, NS, false, false, true>(P, S, src, st, step);
}

// Energy (1/2) c_j^2 |e_i|^2 g of the stored populations: every population of a gas node
// and the emissions of a wall node (the directions towards its gas neighbours).
__global__ void pop_energy_kernel(DevParams P, const float* __restrict__ h, const uint32_t* __restrict__ code,
                                  double* __restrict__ out) {
  __shared__ double sh[8];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double E = 0.0;
  if (n < P.n) {
    const int k = pad_index(P, n % P.nx, n / P.nx);
    const uint32_t cw = code[k];
    const uint32_t c = node_class(cw);
    if (c == GAS || c == WALL) {
      for (int i = 1; i < Q; ++i) {
        if (c == WALL && stencil_of(cw, OPP(i)) == ST_NOT_ARRIVAL) continue;
        const int e2 = EX(i) * EX(i) + EY(i) * EY(i);
        for (int j = 0; j < P.ns; ++j)
          E += eps_weight(P, j, e2) *
               (double(h[(long long)(j * Q + i) * P.plane + k]) + double(P.rref[j]) * double(P.W0[i]));
      }
    }
  }
  const double s = block_sum(E, sh);
  if (threadIdx.x == 0) atomicAdd(out, s);
}
}  // namespace

cudaError_t launch_step_detail(const DevParams& P, const DevState& S, int src, cudaStream_t st, uint32_t step) {
  switch (P.ns) {
    case 1: return detail_ns<1>(P, S, src, st, step);
    case 2: return detail_ns<2>(P, S, src, st, step);
    case 3: return detail_ns<3>(P, S, src, st, step);
    case 4: return detail_ns<4>(P, S, src, st, step);
    case 5: return detail_ns<5>(P, S, src, st, step);
    case 6: return detail_ns<6>(P, S, src, st, step);
    default: return cudaErrorInvalidValue;
  }
}

// D3Q19 inventory (fdlbm3d_ledger_detail.cu).
cudaError_t launch_pop_energy3(const DevParams& P, const DevState& S, int cur, double* out, cudaStream_t st);

cudaError_t launch_pop_energy(const DevParams& P, const DevState& S, int cur, double* out, cudaStream_t st) {
  if (P.dim == 3) return launch_pop_energy3(P, S, cur, out, st);
  if (P.storage != FDLBM_STORAGE_FP32) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  pop_energy_kernel<<<(P.n + 255) / 256, 256, 0, st>>>(P, static_cast<const float*>(S.h[cur]), S.code, out);
  return cudaGetLastError();
}

}  // namespace fdlbm
