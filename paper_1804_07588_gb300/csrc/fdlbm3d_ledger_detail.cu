// D3Q19 step kernels that also keep the exact accounts of the scheme (FP32 population
// storage), and the energy inventory of the stored populations: the D2Q9 accounts of
// fdlbm_ledger_detail.cu on 19 directions. Its own translation unit, so that the
// library's translation units compile in parallel.
#include "fdlbm3d_device.cuh"

namespace fdlbm {

namespace {
template <int NS>
cudaError_t detail3_ns(const DevParams& P, const DevState& S, int src, cudaStream_t st, uint32_t step) {
  return P.energy_correction ? step3_launch<float, NS, true, true>(P, S, src, false, st, step)
                             : step3_launch<float, NS, false, true>(P, S, src, false, st, step);
}

// Energy (1/2) c_j^2 |e_i|^2 g of every population of a gas node and of the emissions of
// a wall node (the directions towards its gas neighbours).
__global__ void pop_energy_kernel3(DevParams P, const float* __restrict__ h, const uint64_t* __restrict__ code,
                                   double* __restrict__ out) {
  __shared__ double sh[8];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double E = 0.0;
  if (n < P.n) {
    int x, y, z;
    xyz_of(P, n, x, y, z);
    const int k = pad3(P, x, y, z);
    const uint64_t cw = code[k];
    const uint32_t c = node_class3(cw);
    if (c == GAS || c == WALL) {
      for (int i = 1; i < Q19; ++i) {
        if (c == WALL && stencil_of3(cw, OPP3(i)) == ST_NOT_ARRIVAL) continue;
        for (int j = 0; j < P.ns; ++j)
          E += eps_weight(P, j, NNZ(i)) *
               (double(h[(long long)(j * Q19 + i) * P.plane + k]) + double(P.rref[j]) * double(P.W0_19[i]));
      }
    }
  }
  const double s = block_sum3(E, sh);
  if (threadIdx.x == 0) atomicAdd(out, s);
}
}  // namespace

cudaError_t launch_step3_detail(const DevParams& P, const DevState& S, int src, cudaStream_t st, uint32_t step) {
  switch (P.ns) {
    case 1: return detail3_ns<1>(P, S, src, st, step);
    case 2: return detail3_ns<2>(P, S, src, st, step);
    case 3: return detail3_ns<3>(P, S, src, st, step);
    case 4: return detail3_ns<4>(P, S, src, st, step);
    case 5: return detail3_ns<5>(P, S, src, st, step);
    case 6: return detail3_ns<6>(P, S, src, st, step);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pop_energy3(const DevParams& P, const DevState& S, int cur, double* out, cudaStream_t st) {
  if (P.storage != FDLBM_STORAGE_FP32) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  pop_energy_kernel3<<<(P.n + 255) / 256, 256, 0, st>>>(P, static_cast<const float*>(S.h[cur]), S.code64, out);
  return cudaGetLastError();
}

}  // namespace fdlbm
