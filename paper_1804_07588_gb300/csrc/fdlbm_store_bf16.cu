// BF16 population storage: instantiates the solver's storage-dependent kernels and
// entry points for __nv_bfloat16 (values rounded once per store; FP32 arithmetic).
#include "fdlbm_device.cuh"

namespace fdlbm {
FDLBM_STORAGE_ENTRY_POINTS(, __nv_bfloat16)
}  // namespace fdlbm
