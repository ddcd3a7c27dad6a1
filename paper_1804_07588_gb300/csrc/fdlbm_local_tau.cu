// D2Q9 step kernels with locally updated relaxation times (Sec. 3: Eqs. tau1s with
// Wilke's mixture rule, tau2_approx_text, D_j_text), FP32 population storage. Their own
// translation unit, so that the library's translation units compile in parallel.
#include "fdlbm_device.cuh"

namespace fdlbm {

namespace {
template <int NS>
cudaError_t local_ns(const DevParams& P, const DevState& S, int src, bool mo, cudaStream_t st, uint32_t step) {
  if (mo)
    return P.energy_correction ? step_launch<float, NS, true, true, false, 1>(P, S, src, st, step)
                               : step_launch<float, NS, false, true, false, 1>(P, S, src, st, step);
  return P.energy_correction ? step_launch<float, NS, true, true>(P, S, src, st, step)
                             : step_launch<float, NS, false, true>(P, S, src, st, step);
}
}  // namespace

cudaError_t launch_step_local_tau(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st,
                                  uint32_t step) {
  switch (P.ns) {
    case 2: return local_ns<2>(P, S, src, moments_only, st, step);
    case 3: return local_ns<3>(P, S, src, moments_only, st, step);
    case 4: return local_ns<4>(P, S, src, moments_only, st, step);
    case 5: return local_ns<5>(P, S, src, moments_only, st, step);
    case 6: return local_ns<6>(P, S, src, moments_only, st, step);
    default: return cudaErrorInvalidValue;  // local relaxation times need >= 2 species
  }
}

}  // namespace fdlbm
