// One persistent launch per step (the batching of Sec. 3.1 taken to a single
// kernel): resets, physics and rendering of every environment in one
// cooperative launch of the rasteriser's persistent grid.
//
//   phase 0  the masked resets: the CTAs stride over the resetting
//            environments, one environment per CTA at a time (the reset's
//            CTA-wide rejection sampling, scratch in global memory per CTA);
//   phase 1  physics: the warps of all CTAs stride over the environments,
//            one warp per environment (the physics kernel's per-warp step,
//            objects staged in the CTA's cluster-list region of shared
//            memory, or in global scratch above 128 objects);
//   phase 2  rendering: the rasteriser's persistent loop, environments pulled
//            from the work counter (costliest scene first when ordered).
//
// A grid-wide barrier separates the phases (physics reads the reset state,
// rendering reads the cameras and objects the physics wrote).  Every CTA is
// resident (cooperative launch with the occupancy-sized grid), and each
// barrier wait is bounded: a wait that gives up sets the device error bit and
// the kernel carries on (the step's results are then wrong, reported as
// GX_EDEVICE; nothing hangs).
#include <math_constants.h>
#include <cuda_fp16.h>

#include "gx_internal.h"
#include "gx_device.cuh"
#include "gx_kin.cuh"
#include "gx_physics_dev.cuh"
#include "gx_raster_dev.cuh"

namespace gx {

namespace {

using namespace rast;

static_assert(GX_MAX_OBJECTS * phys::kTryWindow + GX_MAX_OBJECTS + GX_MAX_OBJECTS / 4 + 1 <=
                  kFusedResetScratch,
              "reset scratch per CTA");

constexpr long kBarrierLimit = 1L << 21;  // polls (about a second) before a barrier wait gives up

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Sense-free grid barrier on two words (arrivals, generation): the last CTA
// to arrive resets the arrival count and advances the generation; the others
// poll the generation, at most kBarrierLimit times.
__device__ void grid_barrier(unsigned* bar, unsigned* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire(bar + 1);
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long it = 0;
      while (ld_acquire(bar + 1) == gen && ++it < kBarrierLimit) {
      }
      if (it >= kBarrierLimit) atomicOr(err, kErrWaitTimeout);
    }
    __threadfence();
  }
  __syncthreads();
}

template <bool kCount>
__global__ void __launch_bounds__(kThreads, kRasterMinBlocks) fused_step_kernel(const FusedParams F) {
  extern __shared__ __align__(128) unsigned char smem[];
  RasterCta<kCount> C;
  uint32_t phase[2];
  Cnt cn;
  raster_cta_begin<kCount>(F.rp, smem, C, phase, cn);
  const int n = F.rp.n, M = F.rp.M;

  // phase 0: masked resets, one environment per CTA at a time
  if (F.reset_mask) {
    float4* scratch = F.reset_scratch + (size_t)blockIdx.x * kFusedResetScratch;
    auto s_cand = reinterpret_cast<float4 (*)[phys::kTryWindow]>(scratch);
    float4* so = scratch + GX_MAX_OBJECTS * phys::kTryWindow;
    float* s_rho = reinterpret_cast<float*>(so + GX_MAX_OBJECTS);
    unsigned* s_bad = reinterpret_cast<unsigned*>(s_rho + GX_MAX_OBJECTS);
    int* s_robot_try = reinterpret_cast<int*>(s_bad + 1);
    for (int env = blockIdx.x; env < n; env += gridDim.x) {
      if (!F.reset_mask[env]) continue;
      phys::reset_env(F.rs, env, s_cand, so, s_rho, *s_bad, *s_robot_try);
      __syncthreads();
    }
    grid_barrier(F.barrier, F.rp.err);
  }

  // phase 1: physics, one warp per environment; the work counter of the
  // rendering phase is zeroed here, before the barrier that orders them
  if (blockIdx.x == 0 && C.tid == 0) *F.rp.work = 0;
  {
    float4* so = M * kWarps <= (int)(kListBytes / sizeof(float4))
                     ? reinterpret_cast<float4*>(C.list) + (size_t)C.warp * M
                     : F.obj_scratch + ((size_t)blockIdx.x * kWarps + C.warp) * GX_MAX_OBJECTS;
    for (int env = blockIdx.x * kWarps + C.warp; env < n; env += gridDim.x * kWarps) {
      phys::physics_env(F.pp, env, C.lane, so);
      __syncwarp();
    }
  }
  grid_barrier(F.barrier, F.rp.err);

  // phase 2: rendering, environments pulled one at a time
  for (;;) {
    if (C.tid == 0) {
      const int k = atomicAdd(F.rp.work, 1);
      C.ctr[0] = (k < n && F.rp.order) ? F.rp.order[k] : k;
    }
    __syncthreads();
    const int env = C.ctr[0];
    if (env >= n) break;
    render_env<kCount, kWarps>(F.rp, env, C, phase, cn);
  }
  raster_cta_end<kCount>(F.rp, C, cn);
}

}  // namespace

cudaError_t fused_configure() {
  const int bytes = (int)raster_smem_bytes(8);
  cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fused_step_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

cudaError_t fused_max_ctas(int* ctas) {
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = fused_configure();
  if (e != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_step_kernel<false>, kThreads,
                                                         raster_smem_bytes(8))) != cudaSuccess)
    return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *ctas = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

cudaError_t launch_fused_step(const FusedParams& f, int ctas, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = raster_smem_bytes(8);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (f.rp.counters) return cudaLaunchKernelEx(&cfg, fused_step_kernel<true>, f);
  return cudaLaunchKernelEx(&cfg, fused_step_kernel<false>, f);
}

}  // namespace gx
