// FP16 population storage of the D3Q19 path: instantiates the storage-dependent 3D
// kernels and entry points for __half (values rounded once per store; FP32 arithmetic).
#include "fdlbm3d_device.cuh"

namespace fdlbm {
FDLBM3_STORAGE_ENTRY_POINTS(, __half)
}  // namespace fdlbm
