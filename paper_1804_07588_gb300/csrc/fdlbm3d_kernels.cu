// D3Q19 path of the solver library: the FP32 instantiation of the 3D kernels and the
// launchers, which dispatch on the population storage type (the BF16 and FP16
// instantiations are in fdlbm3d_store_bf16.cu and fdlbm3d_store_fp16.cu).
#include "fdlbm3d_device.cuh"

namespace fdlbm {

FDLBM3_STORAGE_ENTRY_POINTS(extern, __nv_bfloat16)
FDLBM3_STORAGE_ENTRY_POINTS(extern, __half)
FDLBM3_STORAGE_ENTRY_POINTS(, float)

cudaError_t launch_step3(const DevParams& P, const DevState& S, int src, bool moments_only, cudaStream_t st,
                         uint32_t step) {
  switch (P.storage) {
    case FDLBM_STORAGE_FP32: return storage3_step<float>(P, S, src, moments_only, st, step);
    case FDLBM_STORAGE_BF16: return storage3_step<__nv_bfloat16>(P, S, src, moments_only, st, step);
    case FDLBM_STORAGE_FP16: return storage3_step<__half>(P, S, src, moments_only, st, step);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_init3(const DevParams& P, const DevState& S, const double* X, const double* u,
                         const double* T_lat, const double* Ts_lat, const double* C, const double* inlet,
                         cudaStream_t st) {
  switch (P.storage) {
    case FDLBM_STORAGE_FP32: return storage3_init<float>(P, S, X, u, T_lat, Ts_lat, C, inlet, st);
    case FDLBM_STORAGE_BF16: return storage3_init<__nv_bfloat16>(P, S, X, u, T_lat, Ts_lat, C, inlet, st);
    case FDLBM_STORAGE_FP16: return storage3_init<__half>(P, S, X, u, T_lat, Ts_lat, C, inlet, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_moments_out3(const DevParams& P, const DevState& S, int cur, float* dst, bool t_dev,
                                cudaStream_t st) {
  moments_out_kernel3<<<(P.n + 255) / 256, 256, 0, st>>>(P, S.mom, S.Ts[cur], S.code64, dst, t_dev ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_populations_out3(const DevParams& P, const DevState& S, int cur, float* dst, cudaStream_t st) {
  switch (P.storage) {
    case FDLBM_STORAGE_FP32: return storage3_populations_out<float>(P, S, cur, dst, st);
    case FDLBM_STORAGE_BF16: return storage3_populations_out<__nv_bfloat16>(P, S, cur, dst, st);
    case FDLBM_STORAGE_FP16: return storage3_populations_out<__half>(P, S, cur, dst, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_totals3(const DevParams& P, const DevState& S, int cur, cudaStream_t st) {
  switch (P.storage) {
    case FDLBM_STORAGE_FP32: return storage3_totals<float>(P, S, cur, st);
    case FDLBM_STORAGE_BF16: return storage3_totals<__nv_bfloat16>(P, S, cur, st);
    case FDLBM_STORAGE_FP16: return storage3_totals<__half>(P, S, cur, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_residual3(const DevParams& P, const DevState& S, int cur, cudaStream_t st) {
  double* out = S.red + totals_count(P.ns);
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * residual_count3(P.ns), st);
  if (e != cudaSuccess) return e;
  residual_kernel3<<<(P.n + 255) / 256, 256, 0, st>>>(P, S.mom, S.Ts[cur], S.code64, S.snap, out);
  return cudaGetLastError();
}

}  // namespace fdlbm
