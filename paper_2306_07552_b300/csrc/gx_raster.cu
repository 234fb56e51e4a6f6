// Batched egocentric depth + RGB rendering (Sec. 3.1: one renderer renders
// every environment into one batched observation tensor that stays on the
// GPU).  A CUDA software rasteriser replaces the paper's Vulkan renderer.
//
// Work item: one CTA per (environment, horizontal band of the image).  The
// band's framebuffer lives in shared memory as 64-bit keys
//     key = (~bits(1/z) << 32) | triangle id,
// so one atomicMin keeps the nearest fragment and breaks exact depth ties
// toward the lower triangle id, independently of visiting order.
//
// Pipeline inside a CTA:
//   1. cull the scene's triangle clusters (meshlets) against the band's view
//      frustum and the cluster normal cone (whole clusters facing away);
//   2. warps pull surviving clusters from a shared queue; lane 0 stages each
//      cluster's vertices and triangles into the warp's shared buffers with
//      bulk asynchronous copies (cp.async.bulk + mbarrier), double-buffered so
//      the next cluster streams in while the current one is rasterised;
//   3. lanes transform and snap vertices to 1/256-pixel fixed point; each
//      lane sets up one triangle: back-face test in world space, near-plane
//      test, integer edge functions with the top-left fill rule, depth plane;
//      small triangles are scanned by their lane (int32 edge functions),
//      large or near-clipped ones by the whole warp (int64 edge functions);
//   4. free objects are instanced icosahedra built in the same buffers;
//   5. the band is resolved (depth = 1 / (1/z), colour by triangle id) and
//      written to HBM with coalesced row-major stores.
//
// Every wait is bounded: a wait that gives up sets an error bit and the warp
// stops using its buffers.
#include <math_constants.h>
#include <cuda_fp16.h>

#include "gx_internal.h"

namespace gx {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 512;       // clusters culled per pass
constexpr long kWaitLimit = 1L << 22;

struct WarpSmem {
  float4 vbuf[2][kMeshletMaxVerts];     // staged world-space vertices
  uint32_t tbuf[2][kMeshletMaxTris];    // staged packed triangles
  float4 vc[kMeshletMaxVerts];          // camera-space xyz (w unused)
  int2 vfix[kMeshletMaxVerts];          // snapped screen coordinates (1/256 px)
  unsigned long long bar[2];            // mbarriers of the two buffers
};

struct Cam {
  float rx, ry, rz, ux, uy, uz, fx, fy, fz, ex, ey, ez;
  float f, cx, cy, near_;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait on an mbarrier phase; false when the limit was reached.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t phase) {
  for (long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ int floor_div256(int a) { return a >> 8; }
__device__ __forceinline__ int ceil_div256(int a) { return -((-a) >> 8); }

__device__ __forceinline__ void frag(unsigned long long* fb, int W, int row0, int i, int j, float A,
                                     float B, float C, const Cam& cm, uint32_t id) {
  float invz = fmaf(A, (float)i + 0.5f - cm.cx, fmaf(B, (float)j + 0.5f - cm.cy, C));
  invz = fmaxf(invz, 1e-30f);
  const unsigned long long key =
      ((unsigned long long)(~__float_as_uint(invz)) << 32) | (unsigned long long)id;
  unsigned long long* slot = fb + (j - row0) * W + i;
  if (key < *slot) atomicMin(slot, key);
}

struct Band {
  int W, row0, row1;  // rows [row0, row1)
  // view-frustum side planes of the band, as slopes x/z and y/z with norms
  float tl, tr, tt, tb, kl, kr, kt, kb;
};

// Bounding sphere (world centre c, radius r) vs the band's frustum.
__device__ __forceinline__ bool sphere_visible(const Cam& cm, const Band& bd, float cx, float cy,
                                               float cz, float r) {
  const float dx = cx - cm.ex, dy = cy - cm.ey, dz = cz - cm.ez;
  const float xc = cm.rx * dx + cm.ry * dy + cm.rz * dz;
  const float yc = cm.ux * dx + cm.uy * dy + cm.uz * dz;
  const float zc = cm.fx * dx + cm.fy * dy + cm.fz * dz;
  if (zc + r < cm.near_) return false;
  if ((xc - bd.tl * zc) * bd.kl < -r) return false;
  if ((bd.tr * zc - xc) * bd.kr < -r) return false;
  if ((bd.tt * zc - yc) * bd.kt < -r) return false;
  if ((yc - bd.tb * zc) * bd.kb < -r) return false;
  return true;
}

// Depth plane of a triangle: 1/z at pixel centre (u, v) equals
// A (u - cx) + B (v - cy) + C, from the world-space plane through P0 with
// normal n (h = n . (P0 - eye) < 0 for a front face).
__device__ __forceinline__ void depth_plane(const Cam& cm, float nx, float ny, float nz, float h,
                                            float& A, float& B, float& C) {
  const float ncx = cm.rx * nx + cm.ry * ny + cm.rz * nz;
  const float ncy = cm.ux * nx + cm.uy * ny + cm.uz * nz;
  const float ncz = cm.fx * nx + cm.fy * ny + cm.fz * nz;
  const float ih = 1.0f / h;
  A = ncx * ih / cm.f;
  B = -ncy * ih / cm.f;
  C = ncz * ih;
}

// One lane scans the pixel rectangle of a small triangle (int32 edges).
__device__ void raster_small(unsigned long long* fb, const Band& bd, const Cam& cm, int2 V0,
                             int2 V1, int2 V2, int ix0, int ix1, int iy0, int iy1, float A,
                             float B, float C, uint32_t id) {
  const int dx0 = V1.x - V0.x, dy0 = V1.y - V0.y;
  const int dx1 = V2.x - V1.x, dy1 = V2.y - V1.y;
  const int dx2 = V0.x - V2.x, dy2 = V0.y - V2.y;
  const int b0 = (dy0 < 0 || (dy0 == 0 && dx0 > 0)) ? 0 : -1;
  const int b1 = (dy1 < 0 || (dy1 == 0 && dx1 > 0)) ? 0 : -1;
  const int b2 = (dy2 < 0 || (dy2 == 0 && dx2 > 0)) ? 0 : -1;
  const int px = ix0 * 256 + 128, py = iy0 * 256 + 128;
  int r0 = dx0 * (py - V0.y) - dy0 * (px - V0.x) + b0;
  int r1 = dx1 * (py - V1.y) - dy1 * (px - V1.x) + b1;
  int r2 = dx2 * (py - V2.y) - dy2 * (px - V2.x) + b2;
  const int sx0 = -dy0 * 256, sx1 = -dy1 * 256, sx2 = -dy2 * 256;
  const int sy0 = dx0 * 256, sy1 = dx1 * 256, sy2 = dx2 * 256;
  for (int j = iy0; j <= iy1; ++j) {
    int e0 = r0, e1 = r1, e2 = r2;
    for (int i = ix0; i <= ix1; ++i) {
      if ((e0 | e1 | e2) >= 0) frag(fb, bd.W, bd.row0, i, j, A, B, C, cm, id);
      e0 += sx0;
      e1 += sx1;
      e2 += sx2;
    }
    r0 += sy0;
    r1 += sy1;
    r2 += sy2;
  }
}

// The whole warp scans one triangle (int64 edges): 8x4 pixel blocks.
__device__ void raster_warp_tri(unsigned long long* fb, const Band& bd, const Cam& cm, int2 V0,
                                int2 V1, int2 V2, float A, float B, float C, uint32_t id,
                                int lane) {
  long long area = (long long)(V1.x - V0.x) * (V2.y - V0.y) - (long long)(V2.x - V0.x) * (V1.y - V0.y);
  if (area == 0) return;
  if (area < 0) {
    const int2 t = V1;
    V1 = V2;
    V2 = t;
  }
  const int xmin = min(V0.x, min(V1.x, V2.x)), xmax = max(V0.x, max(V1.x, V2.x));
  const int ymin = min(V0.y, min(V1.y, V2.y)), ymax = max(V0.y, max(V1.y, V2.y));
  const int ix0 = max(ceil_div256(xmin - 128), 0), ix1 = min(floor_div256(xmax - 128), bd.W - 1);
  const int iy0 = max(ceil_div256(ymin - 128), bd.row0);
  const int iy1 = min(floor_div256(ymax - 128), bd.row1 - 1);
  if (ix0 > ix1 || iy0 > iy1) return;
  const int dx0 = V1.x - V0.x, dy0 = V1.y - V0.y;
  const int dx1 = V2.x - V1.x, dy1 = V2.y - V1.y;
  const int dx2 = V0.x - V2.x, dy2 = V0.y - V2.y;
  const long long b0 = (dy0 < 0 || (dy0 == 0 && dx0 > 0)) ? 0 : -1;
  const long long b1 = (dy1 < 0 || (dy1 == 0 && dx1 > 0)) ? 0 : -1;
  const long long b2 = (dy2 < 0 || (dy2 == 0 && dx2 > 0)) ? 0 : -1;
  const int lx = lane & 7, ly = lane >> 3;
  for (int by = iy0; by <= iy1; by += 4) {
    const int j = by + ly;
    for (int bx = ix0; bx <= ix1; bx += 8) {
      const int i = bx + lx;
      if (i > ix1 || j > iy1) continue;
      const long long px = (long long)i * 256 + 128, py = (long long)j * 256 + 128;
      const long long e0 = (long long)dx0 * (py - V0.y) - (long long)dy0 * (px - V0.x) + b0;
      const long long e1 = (long long)dx1 * (py - V1.y) - (long long)dy1 * (px - V1.x) + b1;
      const long long e2 = (long long)dx2 * (py - V2.y) - (long long)dy2 * (px - V2.x) + b2;
      if ((e0 | e1 | e2) >= 0) frag(fb, bd.W, bd.row0, i, j, A, B, C, cm, id);
    }
  }
}

__device__ __forceinline__ int2 project_fix(const Cam& cm, float xc, float yc, float zc) {
  const float iz = __frcp_rn(zc);
  const float px = fminf(fmaxf(xc * iz, -1000.f), 1000.f);
  const float py = fminf(fmaxf(yc * iz, -1000.f), 1000.f);
  return make_int2(__float2int_rn(fmaf(cm.f, px, cm.cx) * 256.f),
                   __float2int_rn(fmaf(-cm.f, py, cm.cy) * 256.f));
}

// Warp-cooperative raster of triangle t of the staged cluster: the whole warp
// recomputes its setup from shared memory, clips it against the near plane
// when needed and scans the (one or two) resulting triangles.
__device__ void raster_big(unsigned long long* fb, const Band& bd, const Cam& cm,
                           const WarpSmem& ws, int buf, uint32_t packed, uint32_t id, int lane) {
  const int i0 = packed & 0xff, i1 = (packed >> 8) & 0xff, i2 = (packed >> 16) & 0xff;
  const float4 P0 = ws.vbuf[buf][i0], P1 = ws.vbuf[buf][i1], P2 = ws.vbuf[buf][i2];
  const float e1x = P1.x - P0.x, e1y = P1.y - P0.y, e1z = P1.z - P0.z;
  const float e2x = P2.x - P0.x, e2y = P2.y - P0.y, e2z = P2.z - P0.z;
  const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
  const float h = nx * (P0.x - cm.ex) + ny * (P0.y - cm.ey) + nz * (P0.z - cm.ez);
  float A, B, C;
  depth_plane(cm, nx, ny, nz, h, A, B, C);
  const float4 v[3] = {ws.vc[i0], ws.vc[i1], ws.vc[i2]};
  const int2 f[3] = {ws.vfix[i0], ws.vfix[i1], ws.vfix[i2]};
  int2 poly[4];
  int m = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 a = v[k], b = v[(k + 1) % 3];
    const bool ain = a.z >= cm.near_, bin = b.z >= cm.near_;
    if (ain) poly[m++] = f[k];
    if (ain != bin) {
      const float t = (cm.near_ - a.z) / (b.z - a.z);
      poly[m++] = project_fix(cm, fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y), cm.near_);
    }
  }
  if (m >= 3) raster_warp_tri(fb, bd, cm, poly[0], poly[1], poly[2], A, B, C, id, lane);
  if (m == 4) raster_warp_tri(fb, bd, cm, poly[0], poly[2], poly[3], A, B, C, id, lane);
}

// Rasterises the cluster staged in buffer `buf` (nv vertices, nt triangles,
// triangle ids id0 + t).
__device__ void raster_cluster(unsigned long long* fb, const Band& bd, const Cam& cm, WarpSmem& ws,
                               int buf, int nv, int nt, uint32_t id0, int small_px, int lane) {
  for (int k = lane; k < nv; k += 32) {
    const float4 P = ws.vbuf[buf][k];
    const float dx = P.x - cm.ex, dy = P.y - cm.ey, dz = P.z - cm.ez;
    const float xc = cm.rx * dx + cm.ry * dy + cm.rz * dz;
    const float yc = cm.ux * dx + cm.uy * dy + cm.uz * dz;
    const float zc = cm.fx * dx + cm.fy * dy + cm.fz * dz;
    ws.vc[k] = make_float4(xc, yc, zc, 0.f);
    ws.vfix[k] = zc >= cm.near_ ? project_fix(cm, xc, yc, zc) : make_int2(0, 0);
  }
  __syncwarp();
  for (int tb = 0; tb < nt; tb += 32) {
    const int t = tb + lane;
    bool big = false;
    uint32_t packed = 0;
    if (t < nt) {
      packed = ws.tbuf[buf][t];
      const int i0 = packed & 0xff, i1 = (packed >> 8) & 0xff, i2 = (packed >> 16) & 0xff;
      const float4 P0 = ws.vbuf[buf][i0], P1 = ws.vbuf[buf][i1], P2 = ws.vbuf[buf][i2];
      const float e1x = P1.x - P0.x, e1y = P1.y - P0.y, e1z = P1.z - P0.z;
      const float e2x = P2.x - P0.x, e2y = P2.y - P0.y, e2z = P2.z - P0.z;
      const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z,
                  nz = e1x * e2y - e1y * e2x;
      const float h = nx * (P0.x - cm.ex) + ny * (P0.y - cm.ey) + nz * (P0.z - cm.ez);
      if (h < 0.f) {  // front-facing
        const float z0 = ws.vc[i0].z, z1 = ws.vc[i1].z, z2 = ws.vc[i2].z;
        const bool c0 = z0 >= cm.near_, c1 = z1 >= cm.near_, c2 = z2 >= cm.near_;
        if (c0 && c1 && c2) {
          int2 V0 = ws.vfix[i0], V1 = ws.vfix[i1], V2 = ws.vfix[i2];
          const long long area = (long long)(V1.x - V0.x) * (V2.y - V0.y) -
                                 (long long)(V2.x - V0.x) * (V1.y - V0.y);
          if (area != 0) {
            if (area < 0) {
              const int2 tmp = V1;
              V1 = V2;
              V2 = tmp;
            }
            const int xmin = min(V0.x, min(V1.x, V2.x)), xmax = max(V0.x, max(V1.x, V2.x));
            const int ymin = min(V0.y, min(V1.y, V2.y)), ymax = max(V0.y, max(V1.y, V2.y));
            const int ix0 = max(ceil_div256(xmin - 128), 0);
            const int ix1 = min(floor_div256(xmax - 128), bd.W - 1);
            const int iy0 = max(ceil_div256(ymin - 128), bd.row0);
            const int iy1 = min(floor_div256(ymax - 128), bd.row1 - 1);
            if (ix0 <= ix1 && iy0 <= iy1) {
              const int npx = (ix1 - ix0 + 1) * (iy1 - iy0 + 1);
              const bool fits32 = (xmax - xmin) < 32768 && (ymax - ymin) < 32768;
              if (fits32 && npx <= small_px) {
                float A, B, C;
                depth_plane(cm, nx, ny, nz, h, A, B, C);
                raster_small(fb, bd, cm, V0, V1, V2, ix0, ix1, iy0, iy1, A, B, C, id0 + t);
              } else {
                big = true;
              }
            }
          }
        } else if (c0 || c1 || c2) {
          big = true;  // crosses the near plane
        }
      }
    }
    unsigned bm = __ballot_sync(kFull, big);
    while (bm) {
      const int L = __ffs(bm) - 1;
      bm &= bm - 1;
      const uint32_t pk = __shfl_sync(kFull, packed, L);
      raster_big(fb, bd, cm, ws, buf, pk, id0 + tb + L, lane);
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kThreads, 2) raster_kernel(const RasterParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int W = P.W, rh = P.region_h;
  unsigned long long* fb = reinterpret_cast<unsigned long long*>(smem);
  uint4* list = reinterpret_cast<uint4*>(smem + (size_t)W * rh * 8);
  int* counters = reinterpret_cast<int*>(list + kChunk);  // [0] count, [1] next
  WarpSmem* wsm = reinterpret_cast<WarpSmem*>(smem + (size_t)W * rh * 8 + kChunk * 16 + 128);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int env = blockIdx.x / P.regions, band = blockIdx.x % P.regions;
  WarpSmem& ws = wsm[warp];
  const DScene& S = P.scenes[P.env_scene[env]];

  Cam cm;
  {
    const float* c = P.cam + (size_t)env * 12;
    cm.rx = c[0]; cm.ux = c[1]; cm.fx = c[2];
    cm.ry = c[3]; cm.uy = c[4]; cm.fy = c[5];
    cm.rz = c[6]; cm.uz = c[7]; cm.fz = c[8];
    cm.ex = c[9]; cm.ey = c[10]; cm.ez = c[11];
    cm.f = 0.5f * (float)W;
    cm.cx = 0.5f * (float)W;
    cm.cy = 0.5f * (float)P.H;
    cm.near_ = P.near_;
  }
  Band bd;
  bd.W = W;
  bd.row0 = band * rh;
  bd.row1 = bd.row0 + rh;
  bd.tl = (-1.f - cm.cx) / cm.f;
  bd.tr = ((float)W + 1.f - cm.cx) / cm.f;
  bd.tt = (cm.cy - ((float)bd.row0 - 1.f)) / cm.f;
  bd.tb = (cm.cy - ((float)bd.row1 + 1.f)) / cm.f;
  bd.kl = rsqrtf(1.f + bd.tl * bd.tl);
  bd.kr = rsqrtf(1.f + bd.tr * bd.tr);
  bd.kt = rsqrtf(1.f + bd.tt * bd.tt);
  bd.kb = rsqrtf(1.f + bd.tb * bd.tb);

  for (int p = tid; p < W * rh; p += kThreads) fb[p] = ~0ull;
  if (lane == 0) {
    mbar_init(&ws.bar[0]);
    mbar_init(&ws.bar[1]);
    fence_mbar_init();
  }
  uint32_t phase[2] = {0u, 0u};
  bool dead = false;  // a wait gave up: this warp stops using its buffers
  __syncthreads();

  for (int base = 0; base < S.n_meshlets; base += kChunk) {
    if (tid == 0) {
      counters[0] = 0;
      counters[1] = 0;
    }
    __syncthreads();
    const int end = min(base + kChunk, S.n_meshlets);
    for (int m = base + tid; m < end; m += kThreads) {
      const float4 h0 = __ldg(S.mhdr + 3 * m), h1 = __ldg(S.mhdr + 3 * m + 1);
      bool vis = sphere_visible(cm, bd, h0.x, h0.y, h0.z, h0.w);
      if (vis) {
        const float4 h2 = __ldg(S.mhdr + 3 * m + 2);
        if (h2.x > -0.5f) {  // normal cone: every face looks away from the eye
          const float vx = h0.x - cm.ex, vy = h0.y - cm.ey, vz = h0.z - cm.ez;
          const float av = h1.x * vx + h1.y * vy + h1.z * vz;
          const float cx_ = h1.y * vz - h1.z * vy, cy_ = h1.z * vx - h1.x * vz,
                      cz_ = h1.x * vy - h1.y * vx;
          const float cr = sqrtf(cx_ * cx_ + cy_ * cy_ + cz_ * cz_);
          if (av * h2.x - cr * h1.w > h0.w * 1.001f + 1e-4f) vis = false;
        }
        if (vis) {
          const int slot = atomicAdd(&counters[0], 1);
          list[slot] = make_uint4(__float_as_uint(h2.y), __float_as_uint(h2.z),
                                  __float_as_uint(h2.w), 0u);
        }
      }
    }
    __syncthreads();
    const int count = counters[0];
    // warps consume the surviving clusters; the next one streams in meanwhile
    int cur = 0, buf = 0;
    if (lane == 0) cur = atomicAdd(&counters[1], 1);
    cur = __shfl_sync(kFull, cur, 0);
    if (!dead && cur < count && lane == 0) {
      const uint4 e = list[cur];
      const int nv = e.z & 0xff, nt = (e.z >> 8) & 0xff;
      const uint32_t tbytes = (uint32_t)((nt + 3) & ~3) * 4u;
      mbar_expect_tx(&ws.bar[0], nv * 16u + tbytes);
      bulk_g2s(ws.vbuf[0], S.mverts + e.x, nv * 16u, &ws.bar[0]);
      bulk_g2s(ws.tbuf[0], S.mtris + e.y, tbytes, &ws.bar[0]);
    }
    while (!dead && cur < count) {
      int nxt = 0;
      if (lane == 0) nxt = atomicAdd(&counters[1], 1);
      nxt = __shfl_sync(kFull, nxt, 0);
      if (nxt < count && lane == 0) {
        const uint4 e = list[nxt];
        const int nv = e.z & 0xff, nt = (e.z >> 8) & 0xff;
        const uint32_t tbytes = (uint32_t)((nt + 3) & ~3) * 4u;
        mbar_expect_tx(&ws.bar[buf ^ 1], nv * 16u + tbytes);
        bulk_g2s(ws.vbuf[buf ^ 1], S.mverts + e.x, nv * 16u, &ws.bar[buf ^ 1]);
        bulk_g2s(ws.tbuf[buf ^ 1], S.mtris + e.y, tbytes, &ws.bar[buf ^ 1]);
      }
      const bool ok = mbar_wait(&ws.bar[buf], phase[buf]);
      phase[buf] ^= 1u;
      if (!__all_sync(kFull, ok)) {
        if (lane == 0) atomicOr(P.err, kErrWaitTimeout);
        // let the copy in flight into the other buffer land before leaving
        if (nxt < count) mbar_wait(&ws.bar[buf ^ 1], phase[buf ^ 1]);
        dead = true;
        break;
      }
      const uint4 e = list[cur];
      raster_cluster(fb, bd, cm, ws, buf, e.z & 0xff, (e.z >> 8) & 0xff, e.y, P.small_px, lane);
      cur = nxt;
      buf ^= 1;
    }
    __syncthreads();
  }

  // free objects: icosahedra scaled to each object's radius
  if (!dead) {
    for (int j = warp; j < P.M; j += kWarps) {
      const float4 o = P.obj[(size_t)env * P.M + j];
      if (!sphere_visible(cm, bd, o.x, o.y, o.z, o.w * 1.0001f + 1e-6f)) continue;
      for (int k = lane; k < P.omesh_nv; k += 32) {
        const float4 u = P.omesh_v[k];
        ws.vbuf[0][k] = make_float4(fmaf(o.w, u.x, o.x), fmaf(o.w, u.y, o.y), fmaf(o.w, u.z, o.z), 0.f);
      }
      for (int k = lane; k < P.omesh_nt; k += 32) ws.tbuf[0][k] = P.omesh_t[k];
      __syncwarp();
      raster_cluster(fb, bd, cm, ws, 0, P.omesh_nv, P.omesh_nt,
                     (uint32_t)S.n_tris + (uint32_t)(j * P.omesh_nt), P.small_px, lane);
    }
  }
  __syncthreads();

  // resolve the band and write it out row-major (coalesced)
  const size_t out0 = ((size_t)env * P.H + bd.row0) * W;
  for (int p = tid; p < W * rh; p += kThreads) {
    const unsigned long long key = fb[p];
    float z = 0.f;
    uint32_t col = 0u;
    if (key != ~0ull) {
      const float invz = __uint_as_float(~(uint32_t)(key >> 32));
      z = 1.0f / invz;
      const uint32_t id = (uint32_t)key;
      col = id < (uint32_t)S.n_tris ? __ldg(S.tri_rgb + id)
                                    : __ldg(P.obj_rgb + (id - (uint32_t)S.n_tris) / P.omesh_nt);
    }
    if (P.depth_fp16)
      reinterpret_cast<__half*>(P.depth)[out0 + p] = __float2half_rn(z);
    else
      reinterpret_cast<float*>(P.depth)[out0 + p] = z;
    if (P.rgb) {
      uint8_t* o = P.rgb + (out0 + p) * 3;
      o[0] = (uint8_t)(col >> 16);
      o[1] = (uint8_t)(col >> 8);
      o[2] = (uint8_t)col;
    }
  }
}

}  // namespace

size_t raster_smem_bytes(int W, int region_h) {
  return (size_t)W * region_h * 8 + kChunk * 16 + 128 + kWarps * sizeof(WarpSmem);
}

cudaError_t raster_configure(int W, int region_h) {
  return cudaFuncSetAttribute(raster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)raster_smem_bytes(W, region_h));
}

void launch_raster(const RasterParams& p, cudaStream_t s) {
  raster_kernel<<<p.n * p.regions, kThreads, raster_smem_bytes(p.W, p.region_h), s>>>(p);
}

}  // namespace gx
