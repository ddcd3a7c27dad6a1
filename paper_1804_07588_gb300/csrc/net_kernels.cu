// Kernels of the learned warm start's network (a 3D U-Net; not in the paper): the 3x3x3
// convolution as an implicit GEMM on the fifth-generation tensor cores, and the small
// layers around it. Activations are NDHWC bf16 (channels innermost, a multiple of 8);
// accumulation is FP32.
//
// conv3_fwd_kernel: one CTA per output tile of 128 voxels (an 8 x 4 x 4 box) and all
// output channels. GEMM D[voxel][o] = sum_k A[voxel][k] B[o][k] with k = (tap, input
// channel): for each of the 27 taps and each input-channel chunk of up to 64, TMA loads
// the input box shifted by the tap (zero fill outside the volume supplies the padding)
// and the weights of that tap, each as 16-byte-wide (8-channel) slabs that land in the
// K-major no-swizzle core-matrix layout, and one thread issues tcgen05.mma (kind::f16,
// bf16 operands) into an FP32 accumulator in tensor memory. A 4-stage ring of shared
// buffers with full/empty mbarriers overlaps loads and MMAs. The epilogue reads the
// accumulator with tcgen05.ld, adds the bias, applies ReLU and/or a ReLU-backward mask,
// and stores bf16. With flipped, transposed weights the same kernel computes the data
// gradient.
// conv3_wgrad_kernel: dW[o][tap][c] = sum_voxels gy[v][o] x[v + tap - 1][c]: a GEMM over
// voxels with both operands MN-major (channels contiguous per voxel, exactly as TMA
// loads them); each CTA reduces a range of voxel tiles into TMEM and adds its partial
// sums into dW with FP32 atomics.
// Every wait on an mbarrier gives up after a time limit, records an error and returns
// (the tensor memory is freed on every path); the host reports the error.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/fdlbm_net.h"

namespace {

constexpr int BX = 8, BY = 4, BZ = 4;  // output tile: 128 voxels
constexpr int TILE_M = 128;
constexpr int STAGES = 4;
constexpr int A_STAGE_BYTES = 8 * TILE_M * 16;  // up to 8 channel groups x 128 rows x 16 B
constexpr int B_STAGE_BYTES = 8 * 128 * 16;     // up to 8 channel groups x 128 rows x 16 B
constexpr long long WAIT_NS = 2000000000LL;     // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes));
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(smem_u32(bar)), "r"(parity));
  return ok != 0;
}
// Wait for the phase of the given parity to complete; false after the time limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try(bar, parity))
    if ((long long)(globaltimer() - t0) > WAIT_NS) return false;
  return true;
}

// TMA tiled loads into shared memory, completing on an mbarrier.
__device__ __forceinline__ void tma_load5(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// tcgen05 shared-memory matrix descriptor, no swizzle: LBO = byte stride between 8-element
// groups along K, SBO = byte stride between 8-row groups along M (or N).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: bf16 A and B, FP32 accumulator, M x N, operand
// majorness (0 K-major, 1 MN-major).
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                   tmem),
               "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols));
}

struct FwdArgs {
  int D, H, W;       // volume (z, y, x)
  int nseg;          // input sources (a concatenation along channels), 1 or 2
  int seg_c[2];      // channels of each source (multiples of 8)
  int cout;          // output channels, a multiple of 16 (<= 128)
  int tmem_cols;
  int a_stage, b_stage;  // bytes of one pipeline stage of the input tile and of the weights,
                         // sized for the largest channel chunk of this call
  int stages;            // halo kernel: stages in the ring (1 or 2)
  const float* bias;  // [cout] or null
  int relu;           // apply ReLU
  const __nv_bfloat16* mask;  // ReLU-backward mask (NDHWC, cout channels) or null
  __nv_bfloat16* y;   // output NDHWC
  int* err;
};

// Input-channel chunks of one tap: (source, first channel, channel count <= 64).
__device__ __forceinline__ int n_chunks(const FwdArgs& a) {
  int n = 0;
  for (int s = 0; s < a.nseg; ++s) n += (a.seg_c[s] + 63) / 64;
  return n;
}
__device__ __forceinline__ void chunk_of(const FwdArgs& a, int q, int& src, int& c0, int& cc, int& woff) {
  woff = 0;
  for (int s = 0; s < a.nseg; ++s) {
    const int nq = (a.seg_c[s] + 63) / 64;
    if (q < nq) {
      src = s;
      c0 = 64 * q;
      cc = min(64, a.seg_c[s] - c0);
      woff += c0;
      return;
    }
    q -= nq;
    woff += a.seg_c[s];
  }
  src = 0, c0 = 0, cc = 0;
}

__global__ void __launch_bounds__(128, 4) conv3_fwd_kernel(const __grid_constant__ CUtensorMap tx0,
                                                           const __grid_constant__ CUtensorMap tx1,
                                                           const __grid_constant__ CUtensorMap tw, FwdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * a.a_stage;
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tslot;
  __shared__ int fail, n_issued, n_used;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // output tile
  const int tiles_x = a.W / BX, tiles_y = a.H / BY, tiles_z = a.D / BZ;
  int t = blockIdx.x;
  const int txi = t % tiles_x;
  t /= tiles_x;
  const int tyi = t % tiles_y;
  t /= tiles_y;
  const int tzi = t % tiles_z;
  const int n = t / tiles_z;
  const int x0 = txi * BX, y0 = tyi * BY, z0 = tzi * BZ;
  const int nq = n_chunks(a);
  const int nstage = 27 * nq;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    fail = 0;
    n_issued = n_used = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) tmem_alloc(&tslot, a.tmem_cols);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      for (int it = 0; it < nstage; ++it) {
        const int s = it % STAGES;
        if (!mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1)) { fail = 1; break; }
        const int tap = it / nq, q = it % nq;
        int src, c0, cc, woff;
        chunk_of(a, q, src, c0, cc, woff);
        const int ng = cc / 8;
        mbar_expect_tx(&full[s], (uint32_t)(ng * (TILE_M * 16 + a.cout * 16)));
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        const CUtensorMap* mx = src == 0 ? &tx0 : &tx1;
        for (int g = 0; g < ng; ++g) {
          tma_load5(sA + s * a.a_stage + g * (TILE_M * 16), mx, c0 + 8 * g, x0 + dx - 1, y0 + dy - 1, z0 + dz - 1, n,
                    &full[s]);
          tma_load3(sB + s * a.b_stage + g * (a.cout * 16), &tw, woff + 8 * g, tap, 0, &full[s]);
        }
        n_issued = it + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = umma_idesc(TILE_M, a.cout, 0, 0);
      for (int it = 0; it < nstage; ++it) {
        const int s = it % STAGES;
        if (!mbar_wait(&full[s], (it / STAGES) & 1)) { fail = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int q = it % nq;
        int src, c0, cc, woff;
        chunk_of(a, q, src, c0, cc, woff);
        const uint32_t abase = smem_u32(sA + s * a.a_stage), bbase = smem_u32(sB + s * a.b_stage);
        for (int k = 0; k < cc / 16; ++k) {
          const uint64_t da = umma_desc(abase + k * 2 * (TILE_M * 16), TILE_M * 16, 128);
          const uint64_t db = umma_desc(bbase + k * 2 * (a.cout * 16), a.cout * 16, 128);
          umma(tmem, da, db, idesc, (it > 0 || k > 0) ? 1u : 0u);
        }
        umma_commit(&empty[s]);
        n_used = it + 1;
      }
      umma_commit(&done);
    }
    __syncwarp();
  }
  // Epilogue: all four warps, warp w reading accumulator lanes 32w..32w+31 (its voxels).
  bool ok = mbar_wait(&done, 0) && !fail;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int r = tid;  // accumulator row = voxel of the tile
    const int x = x0 + r % BX, y = y0 + (r / BX) % BY, z = z0 + r / (BX * BY);
    const long long v = (((long long)n * a.D + z) * a.H + y) * a.W + x;
    __nv_bfloat16* out = a.y + v * a.cout;
    const __nv_bfloat16* mk = a.mask ? a.mask + v * a.cout : nullptr;
    for (int c = 0; c < a.cout; c += 16) {
      float f[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, f);
      __align__(16) __nv_bfloat16 o[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float val = f[i] + (a.bias ? a.bias[c + i] : 0.f);
        if (a.relu) val = fmaxf(val, 0.f);
        if (mk && !(__bfloat162float(mk[c + i]) > 0.f)) val = 0.f;
        o[i] = __float2bfloat16_rn(val);
      }
      reinterpret_cast<uint4*>(out + c)[0] = reinterpret_cast<const uint4*>(o)[0];
      reinterpret_cast<uint4*>(out + c)[1] = reinterpret_cast<const uint4*>(o)[1];
    }
  } else if (tid == 0) {
    atomicExch(a.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  // after a failure, wait (bounded) for loads still in flight into stages nobody consumed
  if (tid == 0)
    for (int it = n_used; it < n_issued; ++it) mbar_wait(&full[it % STAGES], (it / STAGES) & 1);
  __syncthreads();
  if (warp == 0) tmem_free(tmem, a.tmem_cols);
}

// conv3_fwd_halo_kernel: the same convolution for volumes whose H is a multiple of 16,
// with the input staged once per channel chunk instead of once per tap. Output tile: 8
// voxels along x times 16 along y (one z plane), M = 128 rows, row group g = y offset, row
// r within it = x offset. For each chunk of 16 input channels TMA loads the tile's input
// box with its one-voxel halo, 10 x 18 x 3 voxels, as two 8-channel slabs laid out
// [z][y][x][8 channels] (one 16-byte row per voxel), and the weights of all 27 taps of the
// chunk; the A operand of tap (dz, dy, dx) is the same slab read from the offset of voxel
// (dx, dy, dz): its 8-row groups (consecutive x) are 128 contiguous bytes, 160 bytes apart
// along y (SBO), the second slab at the slab stride (LBO). So one load of the halo feeds 27
// MMAs. Stages: a ring of `stages` chunks (1 or 2).
constexpr int HX = 8, HY = 16;               // halo-kernel output tile (x, y)
constexpr int HALO_ROWS = (HX + 2) * (HY + 2) * 3;  // 540 voxels of the halo box
constexpr int HALO_SLAB = (HALO_ROWS * 16 + 127) / 128 * 128;  // bytes per 8-channel slab, 128-B aligned

__global__ void __launch_bounds__(128, 4) conv3_fwd_halo_kernel(const __grid_constant__ CUtensorMap tx0,
                                                                const __grid_constant__ CUtensorMap tx1,
                                                                const __grid_constant__ CUtensorMap tw, FwdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // stage s: A slabs at smem + s * a.a_stage, B (27 taps x cout rows per slab) after the A
  // stages at + s * a.b_stage
  uint8_t* sA = smem;
  uint8_t* sB = smem + a.stages * a.a_stage;
  __shared__ __align__(8) uint64_t full[2], empty[2], done;
  __shared__ uint32_t tslot;
  __shared__ int fail, n_issued, n_used;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = a.W / HX, tiles_y = a.H / HY;
  int t = blockIdx.x;
  const int txi = t % tiles_x;
  t /= tiles_x;
  const int tyi = t % tiles_y;
  t /= tiles_y;
  const int z0 = t % a.D;
  const int n = t / a.D;
  const int x0 = txi * HX, y0 = tyi * HY;
  // chunks of 16 channels over the sources
  int nq = 0;
  for (int s2 = 0; s2 < a.nseg; ++s2) nq += a.seg_c[s2] / 16;
  const int ST = a.stages;
  if (tid == 0) {
    for (int s2 = 0; s2 < ST; ++s2) {
      mbar_init(&full[s2], 1);
      mbar_init(&empty[s2], 1);
    }
    mbar_init(&done, 1);
    fail = 0;
    n_issued = n_used = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) tmem_alloc(&tslot, a.tmem_cols);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  const uint32_t bslab = 27u * (uint32_t)a.cout * 16u;  // bytes of one weight slab (all taps)

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      for (int it = 0; it < nq; ++it) {
        const int s2 = it % ST;
        if (!mbar_wait(&empty[s2], ((it / ST) & 1) ^ 1)) { fail = 1; break; }
        // chunk it: source and first channel, weight column offset
        int q = it, src = 0, c0 = 0, woff = 0;
        for (int g = 0; g < a.nseg; ++g) {
          const int ng = a.seg_c[g] / 16;
          if (q < ng) { src = g; c0 = 16 * q; woff += c0; break; }
          q -= ng;
          woff += a.seg_c[g];
        }
        mbar_expect_tx(&full[s2], 2u * (uint32_t)(HALO_ROWS * 16) + 2u * bslab);
        const CUtensorMap* mx = src == 0 ? &tx0 : &tx1;
        for (int g = 0; g < 2; ++g) {
          tma_load5(sA + s2 * a.a_stage + g * HALO_SLAB, mx, c0 + 8 * g, x0 - 1, y0 - 1, z0 - 1, n, &full[s2]);
          tma_load3(sB + s2 * a.b_stage + g * bslab, &tw, woff + 8 * g, 0, 0, &full[s2]);
        }
        n_issued = it + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer: 27 taps per chunk
      const uint32_t idesc = umma_idesc(128, a.cout, 0, 0);
      for (int it = 0; it < nq; ++it) {
        const int s2 = it % ST;
        if (!mbar_wait(&full[s2], (it / ST) & 1)) { fail = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t abase = smem_u32(sA + s2 * a.a_stage), bbase = smem_u32(sB + s2 * a.b_stage);
        for (int tap = 0; tap < 27; ++tap) {
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          const uint32_t aoff = (uint32_t)(((dz * (HY + 2) + dy) * (HX + 2) + dx) * 16);
          const uint64_t da = umma_desc(abase + aoff, HALO_SLAB, (HX + 2) * 16);
          const uint64_t db = umma_desc(bbase + (uint32_t)tap * (uint32_t)a.cout * 16u, bslab, 128);
          umma(tmem, da, db, idesc, (it > 0 || tap > 0) ? 1u : 0u);
        }
        umma_commit(&empty[s2]);
        n_used = it + 1;
      }
      umma_commit(&done);
    }
    __syncwarp();
  }
  // Epilogue: warp w reads accumulator lanes 32w..32w+31; row r = (y offset) * 8 + x offset.
  bool ok = mbar_wait(&done, 0) && !fail;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int r = tid;
    const int x = x0 + r % HX, y = y0 + r / HX;
    const long long v = (((long long)n * a.D + z0) * a.H + y) * a.W + x;
    __nv_bfloat16* out = a.y + v * a.cout;
    const __nv_bfloat16* mk = a.mask ? a.mask + v * a.cout : nullptr;
    for (int c = 0; c < a.cout; c += 16) {
      float f[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, f);
      __align__(16) __nv_bfloat16 o[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float val = f[i] + (a.bias ? a.bias[c + i] : 0.f);
        if (a.relu) val = fmaxf(val, 0.f);
        if (mk && !(__bfloat162float(mk[c + i]) > 0.f)) val = 0.f;
        o[i] = __float2bfloat16_rn(val);
      }
      reinterpret_cast<uint4*>(out + c)[0] = reinterpret_cast<const uint4*>(o)[0];
      reinterpret_cast<uint4*>(out + c)[1] = reinterpret_cast<const uint4*>(o)[1];
    }
  } else if (tid == 0) {
    atomicExch(a.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0)
    for (int it = n_used; it < n_issued; ++it) mbar_wait(&full[it % ST], (it / ST) & 1);
  __syncthreads();
  if (warp == 0) tmem_free(tmem, a.tmem_cols);
}

struct WgradArgs {
  int D, H, W, N;
  int nseg;
  int seg_c[2];
  int cin;           // total input channels (row length of dW)
  int cout;          // gradient channels (<= 128; padded to M = 128)
  int tiles_per_cta;
  int stages;        // pipeline stages (<= STAGES)
  int b_stage;       // bytes of one input-tile stage (the channel chunk's slabs)
  float* gw;         // [cout][27][cin], accumulated
  int* err;
};

// grid: x = tap (27) x chunk, y = split over voxel tiles
__global__ void __launch_bounds__(128, 3) conv3_wgrad_kernel(const __grid_constant__ CUtensorMap tx0,
                                                             const __grid_constant__ CUtensorMap tx1,
                                                             const __grid_constant__ CUtensorMap tg, WgradArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;                             // gradient tile: 16 channel groups x 128 voxels x 16 B
  uint8_t* sB = smem + a.stages * (16 * TILE_M * 16);  // input tile: the chunk's channel groups
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tslot;
  __shared__ int fail, n_issued, n_used;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int nq = 0;
  for (int s = 0; s < a.nseg; ++s) nq += (a.seg_c[s] + 63) / 64;
  const int tap = blockIdx.x / nq, q = blockIdx.x % nq;
  // chunk of this CTA
  int src = 0, c0 = 0, cc = 0, woff = 0;
  {
    int qq = q;
    for (int s = 0; s < a.nseg; ++s) {
      const int nqs = (a.seg_c[s] + 63) / 64;
      if (qq < nqs) {
        src = s;
        c0 = 64 * qq;
        cc = min(64, a.seg_c[s] - c0);
        woff += c0;
        break;
      }
      qq -= nqs;
      woff += a.seg_c[s];
    }
  }
  const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
  const int tiles_x = a.W / BX, tiles_y = a.H / BY, tiles_z = a.D / BZ;
  const int total_tiles = tiles_x * tiles_y * tiles_z * a.N;
  const int t_first = blockIdx.y * a.tiles_per_cta;
  const int t_last = min(total_tiles, t_first + a.tiles_per_cta);
  const int nstage = max(0, t_last - t_first);
  const int gA = (a.cout + 7) / 8, gB = cc / 8;
  // the gradient operand is padded to 128 rows with zeros that no load overwrites
  for (int i = tid; i < a.stages * 16 * TILE_M * 16 / 16; i += blockDim.x) reinterpret_cast<uint4*>(sA)[i] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;");
  const int ST = a.stages;
  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    fail = 0;
    n_issued = n_used = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) tmem_alloc(&tslot, 64);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  const CUtensorMap* mx = src == 0 ? &tx0 : &tx1;
  if (warp == 0) {
    if (lane == 0) {
      for (int it = 0; it < nstage; ++it) {
        const int s = it % ST;
        if (!mbar_wait(&empty[s], ((it / ST) & 1) ^ 1)) { fail = 1; break; }
        int tt = t_first + it;
        const int txi = tt % tiles_x;
        tt /= tiles_x;
        const int tyi = tt % tiles_y;
        tt /= tiles_y;
        const int tzi = tt % tiles_z;
        const int n = tt / tiles_z;
        const int x0 = txi * BX, y0 = tyi * BY, z0 = tzi * BZ;
        mbar_expect_tx(&full[s], (uint32_t)((gA + gB) * TILE_M * 16));
        for (int g = 0; g < gA; ++g)
          tma_load5(sA + s * (16 * TILE_M * 16) + g * (TILE_M * 16), &tg, 8 * g, x0, y0, z0, n, &full[s]);
        for (int g = 0; g < gB; ++g)
          tma_load5(sB + s * a.b_stage + g * (TILE_M * 16), mx, c0 + 8 * g, x0 + dx - 1, y0 + dy - 1, z0 + dz - 1,
                    n, &full[s]);
        n_issued = it + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = umma_idesc(TILE_M, cc, 1, 1);
      for (int it = 0; it < nstage; ++it) {
        const int s = it % ST;
        if (!mbar_wait(&full[s], (it / ST) & 1)) { fail = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t abase = smem_u32(sA + s * (16 * TILE_M * 16)), bbase = smem_u32(sB + s * a.b_stage);
        // K = voxels: 8 MMAs of 16 voxels; an 8-voxel group is 128 B within a channel slab
        for (int k = 0; k < TILE_M / 16; ++k) {
          const uint64_t da = umma_desc(abase + k * 256, 128, TILE_M * 16);
          const uint64_t db = umma_desc(bbase + k * 256, 128, TILE_M * 16);
          umma(tmem, da, db, idesc, (it > 0 || k > 0) ? 1u : 0u);
        }
        umma_commit(&empty[s]);
        n_used = it + 1;
      }
      umma_commit(&done);
    }
    __syncwarp();
  }
  bool ok = mbar_wait(&done, 0) && !fail;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && nstage > 0) {
    const int o = tid;  // accumulator row = gradient channel
    for (int c = 0; c < cc; c += 16) {
      float f[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, f);
      if (o < a.cout) {
        float* dst = a.gw + ((long long)o * 27 + tap) * a.cin + woff + c;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (c + i < cc) atomicAdd(dst + i, f[i]);
      }
    }
  } else if (!ok && tid == 0) {
    atomicExch(a.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0)
    for (int it = n_used; it < n_issued; ++it) mbar_wait(&full[it % ST], (it / ST) & 1);
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 64);
}

// conv3_wgrad_halo_kernel: the weight gradient for volumes with H a multiple of 16 and a
// 16-channel input chunk per CTA, all 27 taps at once. The accumulators of the taps sit
// side by side in tensor memory (tap t: columns 16 t .. 16 t + 15, 432 of 512). Per voxel
// tile (8 x 16 x 1, voxel k = 8 y + x) TMA loads the output gradient (MN-major A: gradient
// channels padded to 128 rows with zeros, 8-voxel K groups 128 B apart) and the input with
// its one-voxel halo (the forward halo kernel's layout); the B operand of tap (dz, dy, dx) is
// the halo read from voxel (dx, dy, dz): an 8-voxel K group is one halo row of 8
// consecutive x (128 contiguous bytes), the next K group 160 bytes on (LBO), the next 8
// channels a slab further (SBO). 27 taps x 8 MMAs per tile; the partial sums of the CTA's
// tiles are added into dW with FP32 atomics.
__global__ void __launch_bounds__(128, 1) conv3_wgrad_halo_kernel(const __grid_constant__ CUtensorMap tx0,
                                                                  const __grid_constant__ CUtensorMap tx1,
                                                                  const __grid_constant__ CUtensorMap tg, WgradArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int A_ST = 16 * TILE_M * 16;          // gradient tile: 16 slabs x 128 voxels x 16 B
  constexpr int B_ST = 2 * HALO_SLAB;             // input halo: 2 slabs
  uint8_t* sA = smem;
  uint8_t* sB = smem + 2 * A_ST;
  __shared__ __align__(8) uint64_t full[2], empty[2], done;
  __shared__ uint32_t tslot;
  __shared__ int fail, n_issued, n_used;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the CTA's 16-channel chunk
  int q = blockIdx.x, src = 0, c0 = 0, woff = 0;
  for (int g = 0; g < a.nseg; ++g) {
    const int ng = a.seg_c[g] / 16;
    if (q < ng) { src = g; c0 = 16 * q; woff += c0; break; }
    q -= ng;
    woff += a.seg_c[g];
  }
  const int tiles_x = a.W / HX, tiles_y = a.H / HY;
  const int total_tiles = tiles_x * tiles_y * a.D * a.N;
  const int t_first = blockIdx.y * a.tiles_per_cta;
  const int t_last = min(total_tiles, t_first + a.tiles_per_cta);
  const int nstage = max(0, t_last - t_first);
  const int gA = (a.cout + 7) / 8;
  for (int i = tid; i < 2 * A_ST / 16; i += blockDim.x) reinterpret_cast<uint4*>(sA)[i] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;");
  if (tid == 0) {
    for (int s2 = 0; s2 < 2; ++s2) {
      mbar_init(&full[s2], 1);
      mbar_init(&empty[s2], 1);
    }
    mbar_init(&done, 1);
    fail = 0;
    n_issued = n_used = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) tmem_alloc(&tslot, 512);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tslot;
  const CUtensorMap* mx = src == 0 ? &tx0 : &tx1;
  if (warp == 0) {
    if (lane == 0) {
      for (int it = 0; it < nstage; ++it) {
        const int s2 = it & 1;
        if (!mbar_wait(&empty[s2], ((it >> 1) & 1) ^ 1)) { fail = 1; break; }
        int tt = t_first + it;
        const int txi = tt % tiles_x;
        tt /= tiles_x;
        const int tyi = tt % tiles_y;
        tt /= tiles_y;
        const int z0 = tt % a.D;
        const int n = tt / a.D;
        const int x0 = txi * HX, y0 = tyi * HY;
        mbar_expect_tx(&full[s2], (uint32_t)(gA * TILE_M * 16 + 2 * HALO_ROWS * 16));
        for (int g = 0; g < gA; ++g)
          tma_load5(sA + s2 * A_ST + g * (TILE_M * 16), &tg, 8 * g, x0, y0, z0, n, &full[s2]);
        for (int g = 0; g < 2; ++g)
          tma_load5(sB + s2 * B_ST + g * HALO_SLAB, mx, c0 + 8 * g, x0 - 1, y0 - 1, z0 - 1, n, &full[s2]);
        n_issued = it + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = umma_idesc(TILE_M, 16, 1, 1);
      for (int it = 0; it < nstage; ++it) {
        const int s2 = it & 1;
        if (!mbar_wait(&full[s2], (it >> 1) & 1)) { fail = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t abase = smem_u32(sA + s2 * A_ST), bbase = smem_u32(sB + s2 * B_ST);
        for (int tap = 0; tap < 27; ++tap) {
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          const uint32_t boff = (uint32_t)(((dz * (HY + 2) + dy) * (HX + 2) + dx) * 16);
          for (int k = 0; k < TILE_M / 16; ++k) {  // K = 16 voxels = two tile rows
            const uint64_t da = umma_desc(abase + k * 256, 128, TILE_M * 16);
            const uint64_t db = umma_desc(bbase + boff + k * 2 * (HX + 2) * 16, (HX + 2) * 16, HALO_SLAB);
            umma(tmem + (uint32_t)(16 * tap), da, db, idesc, (it > 0 || k > 0) ? 1u : 0u);
          }
        }
        umma_commit(&empty[s2]);
        n_used = it + 1;
      }
      umma_commit(&done);
    }
    __syncwarp();
  }
  bool ok = mbar_wait(&done, 0) && !fail;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && nstage > 0) {
    const int o = tid;  // accumulator row = gradient channel
    for (int tap = 0; tap < 27; ++tap) {
      float f[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * tap), f);
      if (o < a.cout) {
        float* dst = a.gw + ((long long)o * 27 + tap) * a.cin + woff;
#pragma unroll
        for (int i = 0; i < 16; ++i) atomicAdd(dst + i, f[i]);
      }
    }
  } else if (!ok && tid == 0) {
    atomicExch(a.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0)
    for (int it = n_used; it < n_issued; ++it) mbar_wait(&full[it & 1], (it >> 1) & 1);
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 512);
}

// ---- small layers (CUDA cores) ---------------------------------------------------------

// y[v][o] (flipped transpose for the data gradient): W'[c][tap][o] = W[o][26 - tap][c]
__global__ void flip_weights_kernel(const __nv_bfloat16* __restrict__ w, int cout, int cin,
                                    __nv_bfloat16* __restrict__ wf) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)cout * 27 * cin;
  if (i >= total) return;
  const int c = int(i % cin);
  const int tap = int((i / cin) % 27);
  const int o = int(i / (27LL * cin));
  wf[((long long)c * 27 + (26 - tap)) * cout + o] = w[i];
}

__global__ void avgpool2_kernel(const __nv_bfloat16* __restrict__ x, int c, int N, int D, int H, int W,
                                __nv_bfloat16* __restrict__ y) {
  // y has dims D/2, H/2, W/2
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int d2 = D / 2, h2 = H / 2, w2 = W / 2;
  const long long total = (long long)N * d2 * h2 * w2 * c;
  if (i >= total) return;
  const int ch = int(i % c);
  long long v = i / c;
  const int xx = int(v % w2);
  v /= w2;
  const int yy = int(v % h2);
  v /= h2;
  const int zz = int(v % d2);
  const int n = int(v / d2);
  float s = 0.f;
  for (int q = 0; q < 8; ++q) {
    const int z = 2 * zz + (q >> 2), yv = 2 * yy + ((q >> 1) & 1), xv = 2 * xx + (q & 1);
    s += __bfloat162float(x[((((long long)n * D + z) * H + yv) * W + xv) * c + ch]);
  }
  y[i] = __float2bfloat16_rn(0.125f * s);
}

// gradient of avgpool2: each fine voxel gets gy / 8 of its coarse voxel (times the
// ReLU-backward mask of the pooled activation when given)
__global__ void avgpool2_bwd_kernel(const __nv_bfloat16* __restrict__ gy, int c, int N, int D, int H, int W,
                                    const __nv_bfloat16* __restrict__ mask, __nv_bfloat16* __restrict__ gx) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)N * D * H * W * c;
  if (i >= total) return;
  const int ch = int(i % c);
  long long v = i / c;
  const int x = int(v % W);
  v /= W;
  const int y = int(v % H);
  v /= H;
  const int z = int(v % D);
  const int n = int(v / D);
  float g = 0.125f * __bfloat162float(gy[((((long long)n * (D / 2) + z / 2) * (H / 2) + y / 2) * (W / 2) + x / 2) * c + ch]);
  if (mask && !(__bfloat162float(mask[i]) > 0.f)) g = 0.f;
  gx[i] = __float2bfloat16_rn(g);
}

// out[v] = [up2(h)[v] (cu channels), skip[v] (cs channels)] on the fine grid D x H x W
__global__ void up2cat_kernel(const __nv_bfloat16* __restrict__ h, int cu, const __nv_bfloat16* __restrict__ skip,
                              int cs, int N, int D, int H, int W, __nv_bfloat16* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int c = cu + cs;
  const long long total = (long long)N * D * H * W * c;
  if (i >= total) return;
  const int ch = int(i % c);
  long long v = i / c;
  const int x = int(v % W);
  v /= W;
  const int y = int(v % H);
  v /= H;
  const int z = int(v % D);
  const int n = int(v / D);
  if (ch < cu)
    out[i] = h[((((long long)n * (D / 2) + z / 2) * (H / 2) + y / 2) * (W / 2) + x / 2) * cu + ch];
  else
    out[i] = skip[((((long long)n * D + z) * H + y) * W + x) * cs + (ch - cu)];
}

// gradient of up2cat: coarse gh[v'] = sum over its 8 fine voxels of g[.][0:cu]; the skip
// part g[v][cu:] is added into gskip; both times the ReLU-backward masks when given
__global__ void up2cat_bwd_coarse_kernel(const __nv_bfloat16* __restrict__ g, int cu, int cs, int N, int D, int H,
                                         int W, const __nv_bfloat16* __restrict__ mask_h,
                                         __nv_bfloat16* __restrict__ gh) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int d2 = D / 2, h2 = H / 2, w2 = W / 2, c = cu + cs;
  const long long total = (long long)N * d2 * h2 * w2 * cu;
  if (i >= total) return;
  const int ch = int(i % cu);
  long long v = i / cu;
  const int xx = int(v % w2);
  v /= w2;
  const int yy = int(v % h2);
  v /= h2;
  const int zz = int(v % d2);
  const int n = int(v / d2);
  float s = 0.f;
  for (int q = 0; q < 8; ++q) {
    const int z = 2 * zz + (q >> 2), y = 2 * yy + ((q >> 1) & 1), x = 2 * xx + (q & 1);
    s += __bfloat162float(g[((((long long)n * D + z) * H + y) * W + x) * c + ch]);
  }
  if (mask_h && !(__bfloat162float(mask_h[i]) > 0.f)) s = 0.f;
  gh[i] = __float2bfloat16_rn(s);
}
__global__ void up2cat_bwd_skip_kernel(const __nv_bfloat16* __restrict__ g, int cu, int cs, long long nvox,
                                       const __nv_bfloat16* __restrict__ mask_s, __nv_bfloat16* __restrict__ gskip) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nvox * cs) return;
  const long long v = i / cs;
  const int ch = int(i % cs);
  float s = __bfloat162float(gskip[i]) + __bfloat162float(g[v * (cu + cs) + cu + ch]);
  if (mask_s && !(__bfloat162float(mask_s[i]) > 0.f)) s = 0.f;
  gskip[i] = __float2bfloat16_rn(s);
}

// 1x1x1 output head: y[v][o] = b[o] + sum_c w[o][c] h[v][c] (FP32 weights and output)
__global__ void conv1_kernel(const __nv_bfloat16* __restrict__ h, int c, const float* __restrict__ w,
                             const float* __restrict__ b, int cout, long long nvox, float* __restrict__ y) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nvox * cout) return;
  const long long v = i / cout;
  const int o = int(i % cout);
  float s = b[o];
  for (int k = 0; k < c; ++k) s = fmaf(w[o * c + k], __bfloat162float(h[v * c + k]), s);
  y[i] = s;
}
// head backward, input gradient (with the ReLU-backward mask of h)
__global__ void conv1_bwd_data_kernel(const float* __restrict__ gy, int cout, const float* __restrict__ w, int c,
                                      const __nv_bfloat16* __restrict__ h, long long nvox,
                                      __nv_bfloat16* __restrict__ gh) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nvox * c) return;
  const long long v = i / c;
  const int k = int(i % c);
  float s = 0.f;
  for (int o = 0; o < cout; ++o) s = fmaf(w[o * c + k], gy[v * cout + o], s);
  if (!(__bfloat162float(h[i]) > 0.f)) s = 0.f;
  gh[i] = __float2bfloat16_rn(s);
}
// head backward, weight and bias gradients: block-reduced over voxels, atomics into gw, gb
__global__ void conv1_bwd_weight_kernel(const float* __restrict__ gy, int cout, const __nv_bfloat16* __restrict__ h,
                                        int c, long long nvox, float* __restrict__ gw, float* __restrict__ gb) {
  // one thread per (o, k) pair of a block-sized voxel chunk
  extern __shared__ float red[];
  const int pairs = cout * (c + 1);
  for (int p = threadIdx.x; p < pairs; p += blockDim.x) red[p] = 0.f;
  __syncthreads();
  const long long v0 = (long long)blockIdx.x * 256, v1 = min(nvox, v0 + 256);
  for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
    const int o = p / (c + 1), k = p % (c + 1);
    float s = 0.f;
    for (long long v = v0; v < v1; ++v) {
      const float hv = k < c ? __bfloat162float(h[v * c + k]) : 1.f;
      s = fmaf(gy[v * cout + o], hv, s);
    }
    red[p] = s;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
    const int o = p / (c + 1), k = p % (c + 1);
    if (k < c) atomicAdd(gw + o * c + k, red[p]);
    else atomicAdd(gb + o, red[p]);
  }
}

// bias gradient of a conv3 layer: gb[o] = sum_v gy[v][o]
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ gy, int cout, long long nvox,
                                 float* __restrict__ gb) {
  const int o = threadIdx.x % cout;
  const int lanes = blockDim.x / cout;
  const int l = threadIdx.x / cout;
  float s = 0.f;
  if (l < lanes)
    for (long long v = (long long)blockIdx.x * lanes + l; v < nvox; v += (long long)gridDim.x * lanes)
      s += __bfloat162float(gy[v * cout + o]);
  if (l < lanes) atomicAdd(gb + o, s);
}

// weighted MSE over voxels and channels: loss = sum w (y - t)^2 / (cout nvox),
// gy = 2 w (y - t) / (cout nvox); FP64 loss accumulation
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ wgt,
                           int cout, long long nvox, double* __restrict__ loss, float* __restrict__ gy) {
  __shared__ double sh[32];
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const double inv_n = 1.0 / (double(cout) * double(nvox));
  double l = 0.0;
  if (i < nvox * cout) {
    const float w = wgt ? wgt[i / cout] : 1.f;
    const float d = y[i] - t[i];
    l = double(w) * double(d) * double(d) * inv_n;
    gy[i] = float(2.0 * double(w) * double(d) * inv_n);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    atomicAdd(loss, s);
  }
}

// Adam (Kingma and Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr mh / (sqrt(vh) + eps)
// with the bias corrections 1 - b^t; refreshes the bf16 copy of the parameters
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long count, float lr, float b1, float b2, float eps, float c1,
                            float c2, __nv_bfloat16* __restrict__ p16) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (p16) p16[i] = __float2bfloat16_rn(pi);
}

// dst += src (bf16)
__global__ void add_kernel(__nv_bfloat16* __restrict__ dst, const __nv_bfloat16* __restrict__ src, long long count) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < count) dst[i] = __float2bfloat16_rn(__bfloat162float(dst[i]) + __bfloat162float(src[i]));
}

// FP32 -> bf16 copy
__global__ void to_bf16_kernel(const float* __restrict__ x, long long count, __nv_bfloat16* __restrict__ y) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < count) y[i] = __float2bfloat16_rn(x[i]);
}

// ---- host: tensor maps, error flag, launches --------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_mu;
thread_local char g_msg[256];

fdlbm_status net_fail(fdlbm_status st, const char* m) {
  std::snprintf(g_msg, sizeof(g_msg), "%s", m);
  return st;
}

bool encode_fn() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

// NDHWC bf16 activation [N][D][H][W][C]: 5-D map {C, W, H, D, N}, box {8, BX, BY, BZ, 1},
// no swizzle, zero fill outside.
bool act_map(CUtensorMap* m, const void* base, int c, int N, int D, int H, int W) {
  const cuuint64_t dims[5] = {(cuuint64_t)c, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)N};
  const cuuint64_t es = 2;
  const cuuint64_t strides[4] = {c * es, (cuuint64_t)W * c * es, (cuuint64_t)H * W * c * es,
                                 (cuuint64_t)D * H * W * c * es};
  const cuuint32_t box[5] = {8, BX, BY, BZ, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
// weights [cout][27][cin] bf16: 3-D map {cin, 27, cout}, box {8, 1, cout}
bool wt_map(CUtensorMap* m, const void* base, int cin, int cout) {
  const cuuint64_t dims[3] = {(cuuint64_t)cin, 27, (cuuint64_t)cout};
  const cuuint64_t strides[2] = {(cuuint64_t)cin * 2, (cuuint64_t)27 * cin * 2};
  const cuuint32_t box[3] = {8, 1, (cuuint32_t)cout};
  const cuuint32_t estr[3] = {1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The halo kernel's maps: the activation box with its one-voxel halo {8, HX + 2, HY + 2,
// 3, 1}, and the weights of all taps of 8 input channels, {cin, cout, 27} with box {8,
// cout, 27}, so that they land tap-major ([tap][o][8 channels]).
bool act_map_halo(CUtensorMap* m, const void* base, int c, int N, int D, int H, int W) {
  const cuuint64_t dims[5] = {(cuuint64_t)c, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)N};
  const cuuint64_t es = 2;
  const cuuint64_t strides[4] = {c * es, (cuuint64_t)W * c * es, (cuuint64_t)H * W * c * es,
                                 (cuuint64_t)D * H * W * c * es};
  const cuuint32_t box[5] = {8, HX + 2, HY + 2, 3, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
// The halo weight-gradient kernel's output-gradient tile, box {8, HX, HY, 1, 1}.
bool act_map_tile(CUtensorMap* m, const void* base, int c, int N, int D, int H, int W) {
  const cuuint64_t dims[5] = {(cuuint64_t)c, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)N};
  const cuuint64_t es = 2;
  const cuuint64_t strides[4] = {c * es, (cuuint64_t)W * c * es, (cuuint64_t)H * W * c * es,
                                 (cuuint64_t)D * H * W * c * es};
  const cuuint32_t box[5] = {8, HX, HY, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
bool wt_map_taps(CUtensorMap* m, const void* base, int cin, int cout) {
  const cuuint64_t dims[3] = {(cuuint64_t)cin, (cuuint64_t)cout, 27};
  const cuuint64_t strides[2] = {(cuuint64_t)27 * cin * 2, (cuuint64_t)cin * 2};
  const cuuint32_t box[3] = {8, (cuuint32_t)cout, 27};
  const cuuint32_t estr[3] = {1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Per-device error flag of the network kernels (a few bytes, allocated on first use).
int* err_flag() {
  static int* flags[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!flags[dev] && cudaMalloc(&flags[dev], sizeof(int)) == cudaSuccess) cudaMemset(flags[dev], 0, sizeof(int));
  return flags[dev];
}

fdlbm_status check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::snprintf(g_msg, sizeof(g_msg), "%s: %s", what, cudaGetErrorString(e));
    return FDLBM_ECUDA;
  }
  return FDLBM_OK;
}

unsigned blocks_for(long long n, int b = 256) { return (unsigned)((n + b - 1) / b); }

bool vol_ok(int N, int D, int H, int W) {
  return N >= 1 && D >= BZ && H >= BY && W >= BX && D % BZ == 0 && H % BY == 0 && W % BX == 0;
}

}  // namespace

extern "C" {

const char* fdlbm_net_last_error(void) { return g_msg; }

fdlbm_status fdlbm_net_check(void* stream) {
  int* f = err_flag();
  if (!f) return net_fail(FDLBM_ECUDA, "no error flag");
  int h = 0;
  if (cudaMemcpyAsync(&h, f, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    return check_launch("network error flag");
  if (h) {
    cudaMemsetAsync(f, 0, sizeof(int), (cudaStream_t)stream);
    cudaStreamSynchronize((cudaStream_t)stream);
    return net_fail(FDLBM_ETIMEOUT, "a tensor-core convolution timed out waiting on its pipeline");
  }
  return FDLBM_OK;
}

fdlbm_status fdlbm_conv3_fwd(const void* x0, int c0, const void* x1, int c1, int N, int D, int H, int W,
                             const void* wt, const float* bias, int cout, int relu, const void* mask, void* y,
                             void* stream) {
  if (!x0 || !wt || !y || (c1 > 0 && !x1)) return net_fail(FDLBM_EINVAL, "conv3_fwd: null tensor");
  if (c0 <= 0 || c0 % 16 || c1 < 0 || c1 % 16) return net_fail(FDLBM_EINVAL, "conv3_fwd: channels must be multiples of 16");
  if (cout < 16 || cout > 128 || cout % 16) return net_fail(FDLBM_EINVAL, "conv3_fwd: cout must be 16..128, a multiple of 16");
  if (!vol_ok(N, D, H, W)) return net_fail(FDLBM_EINVAL, "conv3_fwd: volume must be a multiple of 4 x 4 x 8 (z, y, x)");
  if (!aligned16(x0) || (x1 && !aligned16(x1)) || !aligned16(wt) || !aligned16(y))
    return net_fail(FDLBM_EINVAL, "conv3_fwd: tensors must be 16-byte aligned");
  if (!encode_fn()) return net_fail(FDLBM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  // the halo kernel for volumes with H a multiple of 16 whose stages fit shared memory
  const int halo_a = 2 * HALO_SLAB, halo_b = 2 * 27 * cout * 16;
  const int halo_chunks = c0 / 16 + c1 / 16;  // 16-channel chunks: one stage each in the ring
  const int halo_stages = (halo_chunks > 1 && 2 * (halo_a + halo_b) <= 200 * 1024) ? 2 : 1;
  const bool halo = H % HY == 0 && W % HX == 0 && halo_stages * (halo_a + halo_b) <= 220 * 1024;
  CUtensorMap m0, m1, mw;
  const bool maps = halo ? (act_map_halo(&m0, x0, c0, N, D, H, W) &&
                            act_map_halo(&m1, c1 > 0 ? x1 : x0, c1 > 0 ? c1 : c0, N, D, H, W) &&
                            wt_map_taps(&mw, wt, c0 + c1, cout))
                         : (act_map(&m0, x0, c0, N, D, H, W) &&
                            act_map(&m1, c1 > 0 ? x1 : x0, c1 > 0 ? c1 : c0, N, D, H, W) && wt_map(&mw, wt, c0 + c1, cout));
  if (!maps) return net_fail(FDLBM_EINVAL, "conv3_fwd: tensor map encoding failed");
  FwdArgs a{};
  a.D = D, a.H = H, a.W = W;
  a.nseg = c1 > 0 ? 2 : 1;
  a.seg_c[0] = c0, a.seg_c[1] = c1;
  a.cout = cout;
  a.tmem_cols = cout <= 32 ? 32 : (cout <= 64 ? 64 : 128);
  a.bias = bias, a.relu = relu;
  a.mask = static_cast<const __nv_bfloat16*>(mask);
  a.y = static_cast<__nv_bfloat16*>(y);
  a.err = err_flag();
  if (!a.err) return net_fail(FDLBM_ECUDA, "conv3_fwd: error flag");
  // stages sized for the largest channel chunk (<= 64 channels), so that small layers
  // leave shared memory for several CTAs per SM
  const int cmax = std::min(64, std::max(c0, c1));
  a.a_stage = (cmax / 8) * TILE_M * 16;
  a.b_stage = (cmax / 8) * cout * 16;
  // Several CTAs share an SM; padding the shared memory keeps their tensor-memory columns
  // within the SM's 512 (228 KB of shared memory per SM: at most 512 / tmem_cols CTAs), so
  // that tcgen05.alloc never has to wait for another CTA's columns.
  const int per_sm = 512 / a.tmem_cols;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(conv3_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         STAGES * (A_STAGE_BYTES + B_STAGE_BYTES));
    cudaFuncSetAttribute(conv3_fwd_halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr = true;
  }
  if (halo) {
    a.a_stage = halo_a;
    a.b_stage = halo_b;
    a.stages = halo_stages;
    const int smem = std::max(halo_stages * (halo_a + halo_b), 233472 / (per_sm + 1) + 1024);
    const unsigned grid = (unsigned)N * D * (H / HY) * (W / HX);
    conv3_fwd_halo_kernel<<<grid, 128, smem, (cudaStream_t)stream>>>(m0, m1, mw, a);
    return check_launch("conv3_fwd");
  }
  const int smem = std::max(STAGES * (a.a_stage + a.b_stage), 233472 / (per_sm + 1) + 1024);
  const unsigned grid = (unsigned)N * (D / BZ) * (H / BY) * (W / BX);
  conv3_fwd_kernel<<<grid, 128, smem, (cudaStream_t)stream>>>(m0, m1, mw, a);
  return check_launch("conv3_fwd");
}

fdlbm_status fdlbm_conv3_flip_weights(const void* wt, int cout, int cin, void* wt_flipped, void* stream) {
  if (!wt || !wt_flipped || cout <= 0 || cin <= 0) return net_fail(FDLBM_EINVAL, "flip_weights: bad arguments");
  const long long total = (long long)cout * 27 * cin;
  flip_weights_kernel<<<blocks_for(total), 256, 0, (cudaStream_t)stream>>>(
      static_cast<const __nv_bfloat16*>(wt), cout, cin, static_cast<__nv_bfloat16*>(wt_flipped));
  return check_launch("flip_weights");
}

fdlbm_status fdlbm_conv3_wgrad(const void* x0, int c0, const void* x1, int c1, int N, int D, int H, int W,
                               const void* gy, int cout, float* gw, float* gb, void* stream) {
  if (!x0 || !gy || !gw || (c1 > 0 && !x1)) return net_fail(FDLBM_EINVAL, "conv3_wgrad: null tensor");
  if (c0 <= 0 || c0 % 16 || c1 < 0 || c1 % 16) return net_fail(FDLBM_EINVAL, "conv3_wgrad: channels must be multiples of 16");
  if (cout < 8 || cout > 128 || cout % 8) return net_fail(FDLBM_EINVAL, "conv3_wgrad: cout must be 8..128, a multiple of 8");
  if (!vol_ok(N, D, H, W)) return net_fail(FDLBM_EINVAL, "conv3_wgrad: volume must be a multiple of 4 x 4 x 8");
  if (!aligned16(x0) || (x1 && !aligned16(x1)) || !aligned16(gy))
    return net_fail(FDLBM_EINVAL, "conv3_wgrad: tensors must be 16-byte aligned");
  if (!encode_fn()) return net_fail(FDLBM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  // the halo kernel (all taps per 16-channel chunk) for volumes with H a multiple of 16
  const bool halo = H % HY == 0 && W % HX == 0;
  CUtensorMap m0, m1, mg;
  const bool maps = halo ? (act_map_halo(&m0, x0, c0, N, D, H, W) &&
                            act_map_halo(&m1, c1 > 0 ? x1 : x0, c1 > 0 ? c1 : c0, N, D, H, W) &&
                            act_map_tile(&mg, gy, cout, N, D, H, W))
                         : (act_map(&m0, x0, c0, N, D, H, W) &&
                            act_map(&m1, c1 > 0 ? x1 : x0, c1 > 0 ? c1 : c0, N, D, H, W) &&
                            act_map(&mg, gy, cout, N, D, H, W));
  if (!maps) return net_fail(FDLBM_EINVAL, "conv3_wgrad: tensor map encoding failed");
  cudaStream_t st = (cudaStream_t)stream;
  const int cin = c0 + c1;
  if (cudaMemsetAsync(gw, 0, sizeof(float) * (size_t)cout * 27 * cin, st) != cudaSuccess)
    return check_launch("conv3_wgrad memset");
  WgradArgs a{};
  if (halo) {
    a.D = D, a.H = H, a.W = W, a.N = N;
    a.nseg = c1 > 0 ? 2 : 1;
    a.seg_c[0] = c0, a.seg_c[1] = c1;
    a.cin = cin, a.cout = cout;
    a.gw = gw;
    a.err = err_flag();
    if (!a.err) return net_fail(FDLBM_ECUDA, "conv3_wgrad: error flag");
    const int tiles = N * D * (H / HY) * (W / HX);
    const int nq = c0 / 16 + c1 / 16;
    // one CTA per SM (it holds all 512 tensor-memory columns): about one wave
    int splits = std::max(1, std::min(tiles, 152 / nq));
    a.tiles_per_cta = (tiles + splits - 1) / splits;
    splits = (tiles + a.tiles_per_cta - 1) / a.tiles_per_cta;
    // two stages of 32 KB + 17 KB, padded so that no second CTA (and tcgen05.alloc of
    // another 512 columns) shares the SM
    const int smem = std::max(2 * (16 * TILE_M * 16 + 2 * HALO_SLAB), 120 * 1024);
    static bool hattr = false;
    if (!hattr) {
      cudaFuncSetAttribute(conv3_wgrad_halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      hattr = true;
    }
    conv3_wgrad_halo_kernel<<<dim3(nq, splits), 128, smem, st>>>(m0, m1, mg, a);
    fdlbm_status s = check_launch("conv3_wgrad");
    if (s != FDLBM_OK || !gb) return s;
    if (cudaMemsetAsync(gb, 0, sizeof(float) * cout, st) != cudaSuccess) return check_launch("bias grad memset");
    const long long nvox = (long long)N * D * H * W;
    bias_grad_kernel<<<std::max(1, std::min(1024, (int)(nvox / 64))), (256 / cout) * cout, 0, st>>>(
        static_cast<const __nv_bfloat16*>(gy), cout, nvox, gb);
    return check_launch("bias grad");
  }
  a.D = D, a.H = H, a.W = W, a.N = N;
  a.nseg = c1 > 0 ? 2 : 1;
  a.seg_c[0] = c0, a.seg_c[1] = c1;
  a.cin = cin, a.cout = cout;
  a.gw = gw;
  a.err = err_flag();
  if (!a.err) return net_fail(FDLBM_ECUDA, "conv3_wgrad: error flag");
  const int tiles = N * (D / BZ) * (H / BY) * (W / BX);
  int nq = (c0 + 63) / 64 + (c1 > 0 ? (c1 + 63) / 64 : 0);
  // about 4 CTAs per SM over taps, chunks and voxel splits
  int splits = std::max(1, std::min(tiles, (152 * 4) / (27 * nq) + 1));
  a.tiles_per_cta = (tiles + splits - 1) / splits;
  splits = (tiles + a.tiles_per_cta - 1) / a.tiles_per_cta;
  // two stages, the input stage sized to the channel chunk: 72-96 KB, two or three CTAs per
  // SM (64 tensor-memory columns each)
  const int cmax = std::min(64, std::max(c0, c1));
  a.stages = 2;
  a.b_stage = (cmax / 8) * TILE_M * 16;
  const int smem = a.stages * (16 * TILE_M * 16 + a.b_stage);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(conv3_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         STAGES * (16 * TILE_M * 16 + A_STAGE_BYTES));
    attr = true;
  }
  conv3_wgrad_kernel<<<dim3(27 * nq, splits), 128, smem, st>>>(m0, m1, mg, a);
  fdlbm_status s = check_launch("conv3_wgrad");
  if (s != FDLBM_OK || !gb) return s;
  if (cudaMemsetAsync(gb, 0, sizeof(float) * cout, st) != cudaSuccess) return check_launch("bias grad memset");
  const long long nvox = (long long)N * D * H * W;
  bias_grad_kernel<<<std::max(1, std::min(1024, (int)(nvox / 64))), (256 / cout) * cout, 0, st>>>(
      static_cast<const __nv_bfloat16*>(gy), cout, nvox, gb);
  return check_launch("bias grad");
}

fdlbm_status fdlbm_net_avgpool2(const void* x, int c, int N, int D, int H, int W, void* y, void* stream) {
  if (!x || !y || D % 2 || H % 2 || W % 2) return net_fail(FDLBM_EINVAL, "avgpool2: bad arguments");
  const long long total = (long long)N * (D / 2) * (H / 2) * (W / 2) * c;
  avgpool2_kernel<<<blocks_for(total), 256, 0, (cudaStream_t)stream>>>(static_cast<const __nv_bfloat16*>(x), c, N, D,
                                                                      H, W, static_cast<__nv_bfloat16*>(y));
  return check_launch("avgpool2");
}

fdlbm_status fdlbm_net_avgpool2_bwd(const void* gy, int c, int N, int D, int H, int W, const void* mask, void* gx,
                                    void* stream) {
  if (!gy || !gx || D % 2 || H % 2 || W % 2) return net_fail(FDLBM_EINVAL, "avgpool2_bwd: bad arguments");
  const long long total = (long long)N * D * H * W * c;
  avgpool2_bwd_kernel<<<blocks_for(total), 256, 0, (cudaStream_t)stream>>>(
      static_cast<const __nv_bfloat16*>(gy), c, N, D, H, W, static_cast<const __nv_bfloat16*>(mask),
      static_cast<__nv_bfloat16*>(gx));
  return check_launch("avgpool2_bwd");
}

fdlbm_status fdlbm_net_up2cat(const void* h, int cu, const void* skip, int cs, int N, int D, int H, int W, void* out,
                              void* stream) {
  if (!h || (cs > 0 && !skip) || cs < 0 || !out || D % 2 || H % 2 || W % 2)
    return net_fail(FDLBM_EINVAL, "up2cat: bad arguments");
  const long long total = (long long)N * D * H * W * (cu + cs);
  up2cat_kernel<<<blocks_for(total), 256, 0, (cudaStream_t)stream>>>(
      static_cast<const __nv_bfloat16*>(h), cu, static_cast<const __nv_bfloat16*>(skip), cs, N, D, H, W,
      static_cast<__nv_bfloat16*>(out));
  return check_launch("up2cat");
}

fdlbm_status fdlbm_net_up2cat_bwd(const void* g, int cu, int cs, int N, int D, int H, int W, const void* mask_h,
                                  void* gh, const void* mask_skip, void* gskip, void* stream) {
  if (!g || !gh || !gskip || D % 2 || H % 2 || W % 2) return net_fail(FDLBM_EINVAL, "up2cat_bwd: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const long long coarse = (long long)N * (D / 2) * (H / 2) * (W / 2) * cu;
  up2cat_bwd_coarse_kernel<<<blocks_for(coarse), 256, 0, st>>>(static_cast<const __nv_bfloat16*>(g), cu, cs, N, D, H,
                                                                W, static_cast<const __nv_bfloat16*>(mask_h),
                                                                static_cast<__nv_bfloat16*>(gh));
  const long long nvox = (long long)N * D * H * W;
  up2cat_bwd_skip_kernel<<<blocks_for(nvox * cs), 256, 0, st>>>(static_cast<const __nv_bfloat16*>(g), cu, cs, nvox,
                                                                 static_cast<const __nv_bfloat16*>(mask_skip),
                                                                 static_cast<__nv_bfloat16*>(gskip));
  return check_launch("up2cat_bwd");
}

fdlbm_status fdlbm_net_conv1(const void* h, int c, const float* w, const float* b, int cout, long long nvox, float* y,
                             void* stream) {
  if (!h || !w || !b || !y) return net_fail(FDLBM_EINVAL, "conv1: null tensor");
  conv1_kernel<<<blocks_for(nvox * cout), 256, 0, (cudaStream_t)stream>>>(static_cast<const __nv_bfloat16*>(h), c, w, b,
                                                                         cout, nvox, y);
  return check_launch("conv1");
}

fdlbm_status fdlbm_net_conv1_bwd(const float* gy, int cout, const float* w, int c, const void* h, long long nvox,
                                 void* gh, float* gw, float* gb, void* stream) {
  if (!gy || !w || !h || !gh || !gw || !gb) return net_fail(FDLBM_EINVAL, "conv1_bwd: null tensor");
  cudaStream_t st = (cudaStream_t)stream;
  conv1_bwd_data_kernel<<<blocks_for(nvox * c), 256, 0, st>>>(gy, cout, w, c, static_cast<const __nv_bfloat16*>(h), nvox,
                                                               static_cast<__nv_bfloat16*>(gh));
  cudaMemsetAsync(gw, 0, sizeof(float) * cout * c, st);
  cudaMemsetAsync(gb, 0, sizeof(float) * cout, st);
  conv1_bwd_weight_kernel<<<blocks_for(nvox, 256), 256, sizeof(float) * cout * (c + 1), st>>>(
      gy, cout, static_cast<const __nv_bfloat16*>(h), c, nvox, gw, gb);
  return check_launch("conv1_bwd");
}

fdlbm_status fdlbm_net_mse(const float* y, const float* t, const float* wgt, int cout, long long nvox, double* loss,
                           float* gy, void* stream) {
  if (!y || !t || !loss || !gy) return net_fail(FDLBM_EINVAL, "mse: null tensor");
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemsetAsync(loss, 0, sizeof(double), st);
  mse_kernel<<<blocks_for(nvox * cout), 256, 0, st>>>(y, t, wgt, cout, nvox, loss, gy);
  return check_launch("mse");
}

fdlbm_status fdlbm_net_adam(float* p, const float* g, float* m, float* v, long long count, int t, float lr, float b1,
                            float b2, float eps, void* p_bf16, void* stream) {
  if (!p || !g || !m || !v || t < 1) return net_fail(FDLBM_EINVAL, "adam: bad arguments");
  const float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
  adam_kernel<<<blocks_for(count), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, count, lr, b1, b2, eps, c1, c2,
                                                                   static_cast<__nv_bfloat16*>(p_bf16));
  return check_launch("adam");
}

fdlbm_status fdlbm_net_add(void* dst, const void* src, long long count, void* stream) {
  if (!dst || !src) return net_fail(FDLBM_EINVAL, "add: null tensor");
  add_kernel<<<blocks_for(count), 256, 0, (cudaStream_t)stream>>>(static_cast<__nv_bfloat16*>(dst),
                                                                 static_cast<const __nv_bfloat16*>(src), count);
  return check_launch("add");
}

fdlbm_status fdlbm_net_to_bf16(const float* x, long long count, void* y, void* stream) {
  if (!x || !y) return net_fail(FDLBM_EINVAL, "to_bf16: null tensor");
  to_bf16_kernel<<<blocks_for(count), 256, 0, (cudaStream_t)stream>>>(x, count, static_cast<__nv_bfloat16*>(y));
  return check_launch("to_bf16");
}

}  // extern "C"
