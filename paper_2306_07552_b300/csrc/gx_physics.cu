// Physics part of the batched step: one warp per environment.
//
// Sec. 3.2 ("Approximate Kinematic Simulation"): action offsets are applied
// directly to the robot state, forward kinematics places the links, the
// candidate pose is tested for overlap with the static scene and the movable
// objects, and any overlap rejects all robot motion for the step.  Grasping
// attaches the object overlapping a small sphere at the end-effector tip; a
// release snaps the object down onto the surface below it and, when that
// fails, restores the object's pre-grasp position (appendix "Object Placing
// Heuristic").  Here the static scene is a signed-distance grid queried by
// trilinear interpolation and free objects are spheres.
//
// Lane layout: lane i < n_spheres carries robot sphere i, lane 30 the held
// object; contact masks are warp ballots, so bit i is lane i.  Every lane
// runs the (cheap) FK chain and keeps only its own link's frame.
#include <math_constants.h>

#include <algorithm>

// This file is compiled twice: as itself (dense grid) and, through
// gx_physics_store.cu, with GX_STATIC_STORE 1 (box store), whose launchers
// carry the suffix _store.
#ifndef GX_STATIC_STORE
#define GX_STATIC_STORE 0
#endif
#if GX_STATIC_STORE == 1
#define GX_LAUNCHER(name) name##_store
#else
#define GX_LAUNCHER(name) name
#endif

#include "gx_internal.h"
#include "gx_device.cuh"
#include "gx_kin.cuh"
#include "gx_physics_dev.cuh"

namespace gx {

namespace {

using namespace phys;

// Seven blocks per SM (72 registers, a few spilled): the kernel waits on
// random grid gathers, and resident warps hide that latency; six blocks (80
// registers), seven and eight (64) measured 0.051, 0.043 and 0.044 ms for
// 4096 environments.
#ifndef GX_PHYS_BLOCKS
#define GX_PHYS_BLOCKS (GX_STATIC_STORE == 1 ? 6 : 7)
#endif
__global__ void __launch_bounds__(32 * kEnvsPerBlock, GX_PHYS_BLOCKS)
    physics_kernel(const PhysicsParams P) {
  __shared__ float4 s_obj[kEnvsPerBlock][GX_MAX_OBJECTS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int env = blockIdx.x * kEnvsPerBlock + w;
  if (blockIdx.x == 0 && threadIdx.x == 0 && P.raster_work && P.nsdf_pass != 1)
    *P.raster_work = 0;
  if (env >= P.n) return;
  physics_env(P, env, lane, s_obj[w]);
}

__global__ void __launch_bounds__(kResetThreads) reset_kernel(const ResetParams P) {
  __shared__ float4 s_cand[GX_MAX_OBJECTS][kTryWindow];  // x, y, z, static test passed
  __shared__ float4 so[GX_MAX_OBJECTS];
  __shared__ float s_rho[GX_MAX_OBJECTS];
  __shared__ unsigned s_bad;
  __shared__ int s_robot_try;
  for (int env = blockIdx.x; env < P.n; env += gridDim.x) {
    if (P.mask && !P.mask[env]) continue;
    reset_env(P, env, s_cand, so, s_rho, s_bad, s_robot_try);
  }
}

// Rebuilds every environment's object broad-phase from the state (after a
// state load): resting objects where they are, a held object where it
// rested before the grasp.
__global__ void bp_rebuild_kernel(const DScene* scenes, const int* env_scene, StateView st, int n,
                                  int M, BpCell* bp, int cells) {
  const int env = blockIdx.x;
  if (env >= n) return;
  const DScene& S = scenes[env_scene[env]];
  BpCell* grids = bp + (size_t)env * 4 * cells;
  uint4* raw = reinterpret_cast<uint4*>(grids);
  for (int i = threadIdx.x; i < 4 * cells; i += blockDim.x) raw[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  const int held = st.held[env];
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const float4 o = st.obj[(size_t)env * M + j];
    float x = o.x, z = o.z;
    if (j == held) {
      x = st.ppre[env];
      z = st.ppre[2 * (size_t)n + env];
    }
    bp_insert(grids, cells, S, j, x, z, o.w);
  }
}

}  // namespace

#if GX_STATIC_STORE == 0
void launch_bp_rebuild(const DScene* scenes, const int* env_scene, const StateView& st, int n,
                       int M, BpCell* bp, int cells, cudaStream_t s) {
  if (n > 0) bp_rebuild_kernel<<<n, 256, 0, s>>>(scenes, env_scene, st, n, M, bp, cells);
}

#endif

void GX_LAUNCHER(launch_physics)(const PhysicsParams& p, cudaStream_t s) {
#if GX_STATIC_STORE == 0
  if (p.store) {
    launch_physics_store(p, s);
    return;
  }
#endif
  const int blocks = (p.n + kEnvsPerBlock - 1) / kEnvsPerBlock;
  physics_kernel<<<blocks, 32 * kEnvsPerBlock, 0, s>>>(p);
}

namespace {
int g_reset_grid = 0;  // CTAs resident at once on this device
}

cudaError_t GX_LAUNCHER(reset_configure)() {
#if GX_STATIC_STORE == 0
  cudaError_t es = reset_configure_store();
  if (es != cudaSuccess) return es;
#endif
  if (g_reset_grid > 0) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reset_kernel, kResetThreads, 0)) !=
          cudaSuccess)
    return e;
  g_reset_grid = std::max(1, sms * per_sm);
  return cudaSuccess;
}

// One wave of resident CTAs striding over the environments: a staggered reset
// of a few environments no longer launches a CTA per environment.
void GX_LAUNCHER(launch_reset)(const ResetParams& p, cudaStream_t s) {
#if GX_STATIC_STORE == 0
  if (p.store) {
    launch_reset_store(p, s);
    return;
  }
#endif
  if (p.n <= 0) return;
  const int grid = std::min(p.n, g_reset_grid > 0 ? g_reset_grid : p.n);
  reset_kernel<<<grid, kResetThreads, 0, s>>>(p);
}

}  // namespace gx
