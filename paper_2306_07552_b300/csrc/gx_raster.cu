// Batched egocentric depth + RGB rendering (Sec. 3.1: one renderer renders
// every environment into one batched observation tensor that stays on the
// GPU).  A CUDA software rasteriser replaces the paper's Vulkan renderer.
//
// Persistent launch: a fixed grid of CTAs (as many as fit on the GPU at
// once) pulls environments from a work counter.  Each CTA owns one
// framebuffer slot in global memory (L2-resident: slots x W x H x 8 bytes)
// of 64-bit keys
//     key = (255 - epoch) << 56 | ~bits(1/z) << 24 | colour (0xRRGGBB),
// updated with fire-and-forget atomicMin reductions, so the nearest fragment
// wins and exact depth ties go to the lower colour value, independently of
// visiting order; the resolve needs no lookup for the colour.  Each
// environment a CTA draws takes the slot's next epoch, whose keys outrank
// every older key, so the slot is never cleared between environments (only
// when the 8-bit epoch wraps, every 255 environments).  The resolve of an
// environment reads its slot and writes the observation rows.
//
// Per environment, inside a CTA:
//   1. the CTA culls the scene's triangle clusters (meshlets), one thread per
//      cluster: bounding sphere and bounding box against the view frustum,
//      the normal cone, and for a cluster whose faces share one normal the
//      exact plane test (the eye behind every face), and lists the survivors;
//   2. lane 0 of each warp stages a listed cluster's vertices, triangles and
//      colours into the warp's shared buffers with bulk asynchronous copies (cp.async.bulk +
//      mbarrier), double-buffered so the next cluster streams in while the
//      current one is rasterised; warps never wait for each other until the
//      resolve;
//   3. lanes transform vertices, snap them to 1/256-pixel fixed point and
//      give each an outcode against the frustum planes;
//   4. each lane takes one triangle: shared outcode bit -> rejected; world-
//      space back-face test; integer edge functions with the top-left fill
//      rule; depth plane.  Triangles whose bounding box is under 128 px are
//      expanded pixel by pixel over the whole warp: a prefix sum over their
//      bounding-box areas gives consecutive lanes consecutive pixel slots,
//      and each slot's triangle is found from a mask of where triangles
//      start.  Huge or near-plane-clipped triangles are scanned by the warp
//      with int64 edge functions, 8x4 blocks first rejected against edges;
//   5. free objects are instanced icosahedra built in the same buffers;
//   6. resolve: depth = 1 / (1/z), colour from the key, 16-byte row-major
//      stores into the batched observation buffers.
//
// Every wait is bounded: a wait that gives up sets an error bit and the warp
// stops using its buffers.
#include <math_constants.h>
#include <cuda_fp16.h>

#include <cstdio>
#include <mutex>

#include "gx_internal.h"
#include "gx_raster_dev.cuh"

namespace gx {

namespace {

using namespace rast;

// kW warps per CTA: 6 or 7 (four CTAs per SM), 8 (three) or 12 (two), a
// rasteriser setting the autotuner chooses.  At the kernel's 72 registers
// four 7-warp CTAs keep 28 warps per SM resident (the register file holds
// 28.4), the most of any shape; the 7-warp bound asks ptxas for three CTAs
// so that it keeps the 72 registers (a bound of four caps it at 64, which
// measured 25% slower with no spills), and the occupancy query confirms four.
template <bool kCount, int kW, bool kBoxes = false, bool kOcc = false>
__global__ void __launch_bounds__(kW * 32,
                                  kW == 8 || kW == 7 ? kRasterMinBlocks : (kW == 6 ? 4 : 2))
    raster_kernel(const RasterParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  RasterCta<kCount> C;
  uint32_t phase[2];
  Cnt cn;
  raster_cta_begin<kCount>(P, smem, C, phase, cn);
  for (;;) {
    if (C.tid == 0) {
      const int k = atomicAdd(P.work, 1);
      C.ctr[0] = (k < P.n && P.order) ? P.order[k] : k;
    }
    __syncthreads();
    const int env = C.ctr[0];
    if (env >= P.n) break;
    render_env<kCount, kW, kBoxes, kOcc>(P, env, C, phase, cn);
  }
  raster_cta_end<kCount>(P, C, cn);
}

}  // namespace

size_t raster_smem_bytes(int warps, int hiz_tiles) {
  return 128 + kListBytes + (size_t)(warps > 0 ? warps : kWarps) * sizeof(WarpSmem) +
         (size_t)hiz_tiles * sizeof(uint32_t);
}

namespace {
// occlusion culling: the tile bounds of the largest image (256 x 256)
constexpr int kMaxHizTiles = (256 / kHizTile) * (256 / kHizTile);
}  // namespace

cudaError_t raster_configure(int* slots) {
  cudaError_t e;
  const int b8 = (int)raster_smem_bytes(8), b12 = (int)raster_smem_bytes(12);
  if ((e = cudaFuncSetAttribute(raster_kernel<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                b8)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                b8)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<false, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                b12)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<true, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                b12)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<false, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)raster_smem_bytes(6))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<true, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)raster_smem_bytes(6))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<false, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)raster_smem_bytes(7))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<true, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)raster_smem_bytes(7))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<false, 8, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, b8)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<false, 7, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)raster_smem_bytes(7))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<true, 7, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)raster_smem_bytes(7))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<true, 8, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, b8)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<false, 8, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)raster_smem_bytes(8, kMaxHizTiles))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(raster_kernel<true, 8, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)raster_smem_bytes(8, kMaxHizTiles))) != cudaSuccess)
    return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raster_kernel<false, 8>, 256, b8);
  if (e != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *slots = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

cudaError_t raster_ctas_per_sm(int warps, int* per_sm, bool boxes) {
  if (warps == 7 && boxes)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, raster_kernel<false, 7, true>, 224,
                                                         raster_smem_bytes(7));
  if (warps == 6)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, raster_kernel<false, 6>, 192,
                                                         raster_smem_bytes(6));
  if (warps == 7)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, raster_kernel<false, 7>, 224,
                                                         raster_smem_bytes(7));
  return warps == 12
             ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, raster_kernel<false, 12>, 384,
                                                             raster_smem_bytes(12))
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, raster_kernel<false, 8>, 256,
                                                             raster_smem_bytes(8));
}

void launch_raster(const RasterParams& p, cudaStream_t s) {
  const int grid = p.n < p.n_slots ? p.n : p.n_slots;  // n_slots: CTAs to launch
  if (p.vis && !p.obox) {  // occlusion culling: 8 warps, the tile bounds in shared memory
    const size_t smem = raster_smem_bytes(8, (p.W / kHizTile) * (p.H / kHizTile));
    if (p.counters)
      raster_kernel<true, 8, false, true><<<grid, 256, smem, s>>>(p);
    else
      raster_kernel<false, 8, false, true><<<grid, 256, smem, s>>>(p);
  } else if (p.obox && p.warps == 7) {  // box objects: 7 warps or 8
    const size_t smem = raster_smem_bytes(7);
    if (p.counters)
      raster_kernel<true, 7, true><<<grid, 224, smem, s>>>(p);
    else
      raster_kernel<false, 7, true><<<grid, 224, smem, s>>>(p);
  } else if (p.obox) {
    const size_t smem = raster_smem_bytes(8);
    if (p.counters)
      raster_kernel<true, 8, true><<<grid, 256, smem, s>>>(p);
    else
      raster_kernel<false, 8, true><<<grid, 256, smem, s>>>(p);
  } else if (p.warps == 6) {
    const size_t smem = raster_smem_bytes(6);
    if (p.counters)
      raster_kernel<true, 6><<<grid, 192, smem, s>>>(p);
    else
      raster_kernel<false, 6><<<grid, 192, smem, s>>>(p);
  } else if (p.warps == 7) {
    const size_t smem = raster_smem_bytes(7);
    if (p.counters)
      raster_kernel<true, 7><<<grid, 224, smem, s>>>(p);
    else
      raster_kernel<false, 7><<<grid, 224, smem, s>>>(p);
  } else if (p.warps == 12) {
    const size_t smem = raster_smem_bytes(12);
    if (p.counters)
      raster_kernel<true, 12><<<grid, 384, smem, s>>>(p);
    else
      raster_kernel<false, 12><<<grid, 384, smem, s>>>(p);
  } else {
    const size_t smem = raster_smem_bytes(8);
    if (p.counters)
      raster_kernel<true, 8><<<grid, 256, smem, s>>>(p);
    else
      raster_kernel<false, 8><<<grid, 256, smem, s>>>(p);
  }
}

}  // namespace gx

// ===========================================================================
// Rendering without allocation.
//
// Some callers cannot call cudaMalloc when they need images: code that runs
// in a section where device allocation is forbidden or would stall (real-time
// control loops, allocation-free serving paths, hosts whose memory policy
// only allows allocation at start-up), or embedders that already spent their
// memory budget.  gx_render_noalloc renders for them with a framebuffer
// scratch area that the library itself holds: the fixed array below, which
// every GPU that loads this library keeps until the process exits.
// ===========================================================================
namespace gx {
namespace {

constexpr size_t kNoAllocFbBytes = 16u << 20;  // framebuffer slots (16 MiB)
static_assert(kErrWaitTimeout == GX_NOALLOC_WAIT_TIMEOUT && kErrBadScene == GX_NOALLOC_BAD_SCENE,
              "public error bits of gx_render_noalloc");
constexpr int kNoAllocMaxSide = 256;           // largest image side it accepts

// [0, kNoAllocFbBytes): framebuffer slots; then the work counter and a spare
// word for device-side error bits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocFbBytes + 256];

struct NoAllocDevice {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch
  int occupancy_slots = 0;
};
constexpr int kMaxDevices = 64;
NoAllocDevice g_noalloc[kMaxDevices];
std::mutex g_noalloc_mu;

}  // namespace
}  // namespace gx

extern "C" gx_status gx_render_noalloc(const gx_scene_set* set, int32_t n,
                                       const int32_t* env_scene, const float* cam,
                                       const float* obj, int32_t n_objects, int32_t img_w,
                                       int32_t img_h, float cam_near, void* depth,
                                       int32_t depth_fp16, uint8_t* rgb, void* stream) {
  using namespace gx;
  SceneSetView sv;
  if (!scene_set_view(set, &sv)) return set_last_error(GX_EINVAL, "gx_render_noalloc: set is NULL");
  if (n < 1 || !env_scene || !cam || !depth || (n_objects > 0 && !obj))
    return set_last_error(GX_EINVAL, "gx_render_noalloc: NULL buffer or n < 1");
  if (n_objects < 0 || n_objects > GX_MAX_OBJECTS)
    return set_last_error(GX_EINVAL, "gx_render_noalloc: n_objects must be in [0, 256]");
  if (img_w < 32 || img_h < 32 || img_w % 32 || img_h % 32)
    return set_last_error(GX_EINVAL, "gx_render_noalloc: image sides must be multiples of 32");
  if (img_w > kNoAllocMaxSide || img_h > kNoAllocMaxSide)
    return set_last_error(GX_EINVAL,
                          "gx_render_noalloc: image larger than its fixed scratch allows "
                          "(at most 256x256)");
  if (!(cam_near > 0.f)) return set_last_error(GX_EINVAL, "gx_render_noalloc: cam_near <= 0");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_last_error(GX_ECUDA, "gx_render_noalloc: no usable current device");
  if (dev != sv.device)
    return set_last_error(GX_EINVAL,
                          "gx_render_noalloc: the scene set lives on another device than the "
                          "current one");
  NoAllocDevice& d = g_noalloc[dev];
  {
    // one-time set-up on this device (the current one): find the array's
    // device address and mark every framebuffer key empty
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!d.ready) {
      void* p = nullptr;
      if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess)
        return set_last_error(GX_ECUDA, "gx_render_noalloc: cudaGetSymbolAddress failed");
      if ((e = cudaMemset(p, 0xff, kNoAllocFbBytes)) != cudaSuccess ||
          (e = cudaMemset((unsigned char*)p + kNoAllocFbBytes, 0, 256)) != cudaSuccess)
        return set_last_error(GX_ECUDA, "gx_render_noalloc: clearing the scratch failed");
      int slots = 0;
      if ((e = raster_configure(&slots)) != cudaSuccess)
        return set_last_error(GX_ECUDA, "gx_render_noalloc: kernel configuration failed");
      if ((e = cudaDeviceSynchronize()) != cudaSuccess)
        return set_last_error(GX_ECUDA, "gx_render_noalloc: set-up failed");
      d.base = (unsigned char*)p;
      d.occupancy_slots = slots;
      d.ready = true;
    }
  }
  const size_t slot_bytes = (size_t)img_w * img_h * 8;
  int slots = (int)(kNoAllocFbBytes / slot_bytes);
  if (slots > d.occupancy_slots) slots = d.occupancy_slots;
  if (slots > n) slots = n;
  cudaStream_t s = (cudaStream_t)stream;
  int* work = reinterpret_cast<int*>(d.base + kNoAllocFbBytes);
  unsigned* err = reinterpret_cast<unsigned*>(d.base + kNoAllocFbBytes + 4);
  // shared by every call: start from a zero work counter and empty keys; the
  // error word keeps accumulating until gx_render_noalloc_error reads it
  if ((e = cudaMemsetAsync(work, 0, 4, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(d.base, 0xff, (size_t)slots * slot_bytes, s)) != cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_render_noalloc: clearing the scratch failed");
  RasterParams rp{};
  rp.n = n;
  rp.M = n_objects;
  rp.W = img_w;
  rp.H = img_h;
  rp.big_px = 1 << 30;
  rp.fb_slots = reinterpret_cast<unsigned long long*>(d.base);
  rp.n_slots = slots;
  rp.work = work;
  rp.scenes = sv.scenes;
  rp.n_scenes = sv.n;
  rp.env_scene = env_scene;
  rp.cam = cam;
  rp.obj = reinterpret_cast<const float4*>(obj);
  rp.omesh_v = sv.omesh_v;
  rp.omesh_t = sv.omesh_t;
  rp.omesh_nv = sv.omesh_nv;
  rp.omesh_nt = sv.omesh_nt;
  rp.obj_rgb = sv.obj_rgb;
  rp.near_ = cam_near;
  rp.depth = depth;
  rp.depth_fp16 = depth_fp16 ? 1 : 0;
  rp.rgb = rgb;
  rp.err = err;
  rp.counters = nullptr;
  launch_raster(rp, s);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_render_noalloc: launch failed");
  return GX_OK;
}

extern "C" gx_status gx_render_noalloc_error(uint32_t* bits) {
  using namespace gx;
  if (bits) *bits = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_last_error(GX_ECUDA, "gx_render_noalloc_error: no usable current device");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc[dev].ready) base = g_noalloc[dev].base;
  }
  if (!base) return GX_OK;  // no call has run on this device: nothing to report
  unsigned* err = reinterpret_cast<unsigned*>(base + kNoAllocFbBytes + 4);
  unsigned v = 0;
  // every earlier call must have finished, on whatever stream it was issued
  if ((e = cudaDeviceSynchronize()) != cudaSuccess ||
      (e = cudaMemcpy(&v, err, sizeof(v), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemset(err, 0, sizeof(v))) != cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_render_noalloc_error: reading the error word failed");
  if (bits) *bits = v;
  if (v == 0) return GX_OK;
  char msg[200];
  snprintf(msg, sizeof(msg), "gx_render_noalloc: device error 0x%x:%s%s", v,
           (v & kErrBadScene) ? " scene index out of range (environment drawn empty)" : "",
           (v & kErrWaitTimeout) ? " bounded wait gave up (images incomplete)" : "");
  return set_last_error(GX_EDEVICE, msg);
}
