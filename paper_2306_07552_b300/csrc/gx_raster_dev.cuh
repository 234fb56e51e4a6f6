// Device code of the persistent software rasteriser (Sec. 3.1), shared by
// its own kernel (gx_raster.cu) and the fused persistent step (gx_fused.cu).
// Each including translation unit gets its own internal copy.
#pragma once

#include <type_traits>

#include <math_constants.h>
#include <cuda_fp16.h>

#include "gx_internal.h"

namespace gx {
namespace {
namespace rast {


constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = kRasterThreads;
constexpr int kWarps = kThreads / 32;
constexpr long kWaitLimit = 1L << 22;  // bounded waits
constexpr int kListCap = 2048;          // clusters culled per pass
// bytes of the CTA's cluster list: one cluster index per entry (the copy
// offsets and counts are read from the cluster's header when it is issued)
constexpr size_t kListBytes = kListCap * sizeof(uint32_t);
constexpr int kSpan = 4;                // adjacent pixels of a row per expansion slot
#ifndef GX_RASTER_DIRECT_W
#define GX_RASTER_DIRECT_W 2
#endif
#ifndef GX_RASTER_DIRECT_H
#define GX_RASTER_DIRECT_H 2
#endif
// bounding boxes up to this size are tested by their set-up lane (no slots)
constexpr int kDirectW = GX_RASTER_DIRECT_W, kDirectH = GX_RASTER_DIRECT_H;
constexpr float kClassPx = 64.f;        // screen radius (pixels) of the costliest cluster class

// The box objects' instance mesh: the unit cube's twelve triangles (corner k
// has the signs of bits 0/1/2 of k on x/y/z), counter-clockwise seen from
// outside, packed i0 | i1 << 8 | i2 << 16.
__constant__ uint32_t kCubeTris[12] = {
    0 | 4 << 8 | 6 << 16, 0 | 6 << 8 | 2 << 16, 1 | 3 << 8 | 7 << 16, 1 | 7 << 8 | 5 << 16,
    0 | 1 << 8 | 5 << 16, 0 | 5 << 8 | 4 << 16, 2 | 6 << 8 | 7 << 16, 2 | 7 << 8 | 3 << 16,
    0 | 2 << 8 | 3 << 16, 0 | 3 << 8 | 1 << 16, 4 | 5 << 8 | 7 << 16, 4 | 7 << 8 | 6 << 16};

// Setup of one triangle queued for pixel expansion.
struct __align__(16) ExpTri {
  int e[3];       // edge values at the bounding box's first pixel centre (bias included)
  int ixy;        // ix0 | iy0 << 16
  int sx[3];      // edge increments per pixel step in x
  int bw;         // bounding-box width in pixels
  int sy[3];      // edge increments per pixel step in y
  uint32_t rgb;   // colour, the key's low word
  float A, B, C;  // 1/z plane
  int off;        // first expansion slot of this round
  float inv_bp;   // 1 / pairs per row
  int pad[3];
};

struct __align__(16) WarpSmem {
  float4 vbuf[2][kMeshletMaxVerts];     // staged world-space vertices
  ExpTri q[32];                         // expansion queue of one round
  uint32_t tbuf[2][kMeshletMaxTris];    // staged packed triangles
  uint32_t cbuf[2][kMeshletMaxTris];    // their colours, 0xRRGGBB
  int2 vfix[kMeshletMaxVerts];          // snapped screen coordinates (1/256 px)
  float vz[kMeshletMaxVerts];           // camera-space depth
  uint8_t voc[kMeshletMaxVerts];        // frustum outcode
  uint8_t qlane[32];                    // lanes whose triangles have pixels, in order
  unsigned long long bar[2];            // mbarriers of the two buffers
  uint2 ent[2];                         // the clusters issued into them (cluster_entry)
};

// Per-lane work counters, summed into RasterParams::counters when counting.
struct Cnt {
  unsigned long long v[kRasterCounters];
};

struct Cam {
  float rx, ry, rz, ux, uy, uz, fx, fy, fz, ex, ey, ez;
  float f, cx, cy, near_;
};

struct View {
  int W, H;
  unsigned long long* fb;  // this CTA's slot, [H][W]
  uint64_t pol;            // L2 policy keeping the slot resident
  unsigned long long tag;  // this environment's epoch field, (255 - epoch) << 56
  // side planes of the frustum as slopes x/z, y/z, with 1/|n|
  float tl, tr, tt, tb, kl, kr, kt, kb;
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
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t phase,
                                          unsigned long long* polls = nullptr) {
  for (long it = 0; it < kWaitLimit; ++it) {
    if (polls) ++*polls;
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

// Depth test of one fragment: invz = 1/z at the pixel centre, key (~bits(invz) << 32) | rgb
// reduced with min into the framebuffer word fbp.
template <bool kCount>
__device__ __forceinline__ void frag_key(const View& vw, unsigned long long* fbp, float invz,
                                         uint32_t rgb, Cnt& cn) {
  if (kCount) cn.v[kCntFragments]++;
  invz = fmaxf(invz, 1e-30f);
  const unsigned long long key =
      vw.tag | ((unsigned long long)(~__float_as_uint(invz)) << 24) | (unsigned long long)rgb;
  // fire-and-forget reduction in L2, the slot marked to stay resident there
  asm volatile("red.relaxed.gpu.global.min.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(fbp),
               "l"(key), "l"(vw.pol)
               : "memory");
}

// Pixel (i, j): the plane A u + B v + C at the pixel centre's offset from the
// principal point.
template <bool kCount>
__device__ __forceinline__ void frag(const View& vw, int i, int j, float A, float B, float C,
                                     const Cam& cm, uint32_t rgb, Cnt& cn) {
  frag_key<kCount>(vw, vw.fb + j * vw.W + i,
                   fmaf(A, (float)i + 0.5f - cm.cx, fmaf(B, (float)j + 0.5f - cm.cy, C)), rgb, cn);
}

// Bounding sphere (world centre c, radius r) vs the view frustum.
__device__ __forceinline__ bool sphere_visible(const Cam& cm, const View& vw, float cx, float cy,
                                               float cz, float r) {
  const float dx = cx - cm.ex, dy = cy - cm.ey, dz = cz - cm.ez;
  const float xc = cm.rx * dx + cm.ry * dy + cm.rz * dz;
  const float yc = cm.ux * dx + cm.uy * dy + cm.uz * dz;
  const float zc = cm.fx * dx + cm.fy * dy + cm.fz * dz;
  if (zc + r < cm.near_) return false;
  if ((xc - vw.tl * zc) * vw.kl < -r) return false;
  if ((vw.tr * zc - xc) * vw.kr < -r) return false;
  if ((vw.tt * zc - yc) * vw.kt < -r) return false;
  if ((yc - vw.tb * zc) * vw.kb < -r) return false;
  return true;
}

// Bounding box (corners lo.xyz, hi.xyz) vs the view frustum: false when all
// its corners lie outside one side plane or in front of the near plane (then
// so do all the cluster's vertices, whose outcodes would reject every
// triangle).  A plane n . (P - eye) >= 0 holds somewhere in the box iff it
// holds at the corner n points to; a small relative margin keeps the test
// conservative against rounding.
__device__ __forceinline__ float plane_max(float nx, float ny, float nz, const Cam& cm, float4 lo,
                                           float4 hi) {
  const float px = nx >= 0.f ? hi.x : lo.x, py = ny >= 0.f ? hi.y : lo.y,
              pz = nz >= 0.f ? hi.z : lo.z;
  return nx * (px - cm.ex) + ny * (py - cm.ey) + nz * (pz - cm.ez);
}

__device__ __forceinline__ bool box_visible(const Cam& cm, const View& vw, float4 lo, float4 hi) {
  const float ext = fabsf(hi.x - cm.ex) + fabsf(hi.y - cm.ey) + fabsf(hi.z - cm.ez) +
                    fabsf(lo.x - cm.ex) + fabsf(lo.y - cm.ey) + fabsf(lo.z - cm.ez);
  const float eps = 1e-5f * ext + 1e-5f;
  // camera axes: right r, up u, forward f (rows of the view rotation)
  if (plane_max(cm.fx, cm.fy, cm.fz, cm, lo, hi) < cm.near_ - eps) return false;
  if (plane_max(cm.rx - vw.tl * cm.fx, cm.ry - vw.tl * cm.fy, cm.rz - vw.tl * cm.fz, cm, lo, hi) <
      -eps * (1.f + fabsf(vw.tl)))
    return false;
  if (plane_max(vw.tr * cm.fx - cm.rx, vw.tr * cm.fy - cm.ry, vw.tr * cm.fz - cm.rz, cm, lo, hi) <
      -eps * (1.f + fabsf(vw.tr)))
    return false;
  if (plane_max(vw.tt * cm.fx - cm.ux, vw.tt * cm.fy - cm.uy, vw.tt * cm.fz - cm.uz, cm, lo, hi) <
      -eps * (1.f + fabsf(vw.tt)))
    return false;
  if (plane_max(cm.ux - vw.tb * cm.fx, cm.uy - vw.tb * cm.fy, cm.uz - vw.tb * cm.fz, cm, lo, hi) <
      -eps * (1.f + fabsf(vw.tb)))
    return false;
  return true;
}

// Reciprocal by the hardware approximation (PTX rcp.approx.f32, within 1 ulp).
// Every use tolerates it: depth-plane coefficients and the resolved depth stay
// within a few ulp (the depth tolerance is 1e-5 relative); a projected vertex
// moves by far less than its 1/256-pixel snapping step; and the row of an
// expansion slot, floor((r + 0.5) / runs), keeps at least 1/128 between its
// argument and an integer for the at most 64 four-pixel runs of a row.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Depth plane of a triangle: 1/z at pixel centre (u, v) equals
// A (u - cx) + B (v - cy) + C, from the world-space plane through P0 with
// normal n (h = n . (P0 - eye) < 0 for a front face).
__device__ __forceinline__ void depth_plane(const Cam& cm, float nx, float ny, float nz, float h,
                                            float& A, float& B, float& C) {
  const float ncx = cm.rx * nx + cm.ry * ny + cm.rz * nz;
  const float ncy = cm.ux * nx + cm.uy * ny + cm.uz * nz;
  const float ncz = cm.fx * nx + cm.fy * ny + cm.fz * nz;
  // one reciprocal: 1/z = (ncx u - ncy v) / (h f) + ncz / h at pixel offset (u, v)
  const float s = rcp_approx(h * cm.f);
  A = ncx * s;
  B = -ncy * s;
  C = (ncz * cm.f) * s;
}

__device__ __forceinline__ int2 project_fix(const Cam& cm, float xc, float yc, float zc) {
  const float iz = rcp_approx(zc);
  const float px = fminf(fmaxf(xc * iz, -1000.f), 1000.f);
  const float py = fminf(fmaxf(yc * iz, -1000.f), 1000.f);
  return make_int2(__float2int_rn(fmaf(cm.f, px, cm.cx) * 256.f),
                   __float2int_rn(fmaf(-cm.f, py, cm.cy) * 256.f));
}

__device__ __forceinline__ bool top_left(int dx, int dy) { return dy < 0 || (dy == 0 && dx > 0); }

// The whole warp scans one triangle with int64 edge functions.  Lanes first
// test 32 8x4 blocks at a time against the three edges (each edge at the
// block corner where it is largest); only blocks no edge excludes are
// scanned, one pixel per lane.
template <bool kCount>
__device__ void raster_warp_tri(const View& vw, const Cam& cm, int2 V0, int2 V1, int2 V2, float A,
                                float B, float C, uint32_t rgb, int lane, Cnt& cn) {
  const long long area =
      (long long)(V1.x - V0.x) * (V2.y - V0.y) - (long long)(V2.x - V0.x) * (V1.y - V0.y);
  if (area == 0) return;
  if (area < 0) {
    const int2 t = V1;
    V1 = V2;
    V2 = t;
  }
  const int xmin = min(V0.x, min(V1.x, V2.x)), xmax = max(V0.x, max(V1.x, V2.x));
  const int ymin = min(V0.y, min(V1.y, V2.y)), ymax = max(V0.y, max(V1.y, V2.y));
  const int ix0 = max(ceil_div256(xmin - 128), 0), ix1 = min(floor_div256(xmax - 128), vw.W - 1);
  const int iy0 = max(ceil_div256(ymin - 128), 0), iy1 = min(floor_div256(ymax - 128), vw.H - 1);
  if (ix0 > ix1 || iy0 > iy1) return;
  const int2 V[3] = {V0, V1, V2};
  int dx[3], dy[3];
  long long b[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dx[k] = V[(k + 1) % 3].x - V[k].x;
    dy[k] = V[(k + 1) % 3].y - V[k].y;
    b[k] = top_left(dx[k], dy[k]) ? 0 : -1;
  }
  const int nbx = (ix1 - ix0) / 8 + 1, nby = (iy1 - iy0) / 4 + 1;
  const int nblk = nbx * nby;
  const int lx = lane & 7, ly = lane >> 3;
  for (int base = 0; base < nblk; base += 32) {
    const int blk = base + lane;
    bool keep = false;
    if (blk < nblk) {
      const int bx = ix0 + (blk % nbx) * 8, by = iy0 + (blk / nbx) * 4;
      const int bx1 = min(bx + 7, ix1), by1 = min(by + 3, iy1);
      keep = true;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const long long px = (long long)(dy[k] < 0 ? bx1 : bx) * 256 + 128;
        const long long py = (long long)(dx[k] > 0 ? by1 : by) * 256 + 128;
        const long long e = (long long)dx[k] * (py - V[k].y) - (long long)dy[k] * (px - V[k].x) + b[k];
        keep &= e >= 0;
      }
    }
    unsigned m = __ballot_sync(kFull, keep);
    while (m) {
      const int L = __ffs(m) - 1;
      m &= m - 1;
      const int blk2 = base + L;
      if (kCount && lane == 0) cn.v[kCntBigBlocks]++;
      const int i = ix0 + (blk2 % nbx) * 8 + lx, j = iy0 + (blk2 / nbx) * 4 + ly;
      if (i > ix1 || j > iy1) continue;
      const long long px = (long long)i * 256 + 128, py = (long long)j * 256 + 128;
      bool in = true;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        in &= (long long)dx[k] * (py - V[k].y) - (long long)dy[k] * (px - V[k].x) + b[k] >= 0;
      if (in) frag<kCount>(vw, i, j, A, B, C, cm, rgb, cn);
    }
  }
}

// Warp-cooperative raster of a triangle of the staged cluster: every lane
// recomputes its setup, clips it against the near plane when needed and the
// warp scans the (one or two) resulting triangles.
template <bool kCount>
__device__ void raster_big(const View& vw, const Cam& cm, const WarpSmem& ws, int buf,
                           uint32_t packed, uint32_t rgb, int lane, Cnt& cn) {
  if (kCount && lane == 0) cn.v[kCntTrisBig]++;
  const int idx[3] = {(int)(packed & 0xff), (int)((packed >> 8) & 0xff), (int)((packed >> 16) & 0xff)};
  const float4 P0 = ws.vbuf[buf][idx[0]], P1 = ws.vbuf[buf][idx[1]], P2 = ws.vbuf[buf][idx[2]];
  const float e1x = P1.x - P0.x, e1y = P1.y - P0.y, e1z = P1.z - P0.z;
  const float e2x = P2.x - P0.x, e2y = P2.y - P0.y, e2z = P2.z - P0.z;
  const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
  const float h = nx * (P0.x - cm.ex) + ny * (P0.y - cm.ey) + nz * (P0.z - cm.ez);
  float A, B, C;
  depth_plane(cm, nx, ny, nz, h, A, B, C);
  float3 v[3];
  int2 f[3];
  bool clipped = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 P = ws.vbuf[buf][idx[k]];
    const float dx = P.x - cm.ex, dy = P.y - cm.ey, dz = P.z - cm.ez;
    v[k] = make_float3(cm.rx * dx + cm.ry * dy + cm.rz * dz, cm.ux * dx + cm.uy * dy + cm.uz * dz,
                       ws.vz[idx[k]]);
    f[k] = ws.vfix[idx[k]];
    clipped |= v[k].z < cm.near_;
  }
  if (kCount && clipped && lane == 0) cn.v[kCntTrisClipped]++;
  int2 poly[4];
  int m = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float3 a = v[k], b = v[(k + 1) % 3];
    const bool ain = a.z >= cm.near_, bin = b.z >= cm.near_;
    if (ain) poly[m++] = f[k];
    if (ain != bin) {
      const float t = (cm.near_ - a.z) / (b.z - a.z);
      poly[m++] = project_fix(cm, fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y), cm.near_);
    }
  }
  if (m >= 3) raster_warp_tri<kCount>(vw, cm, poly[0], poly[1], poly[2], A, B, C, rgb, lane, cn);
  if (m == 4) raster_warp_tri<kCount>(vw, cm, poly[0], poly[2], poly[3], A, B, C, rgb, lane, cn);
}

// Rasterises the cluster staged in buffer `buf` (nv vertices, nt triangles
// with their colours).
template <bool kCount>
__device__ void raster_cluster(const View& vw, const Cam& cm, WarpSmem& ws, int buf, int nv, int nt,
                               int big_px, int lane, Cnt& cn) {
  if (kCount && lane == 0) cn.v[kCntClustersDrawn]++;
  for (int k = lane; k < nv; k += 32) {
    const float4 P = ws.vbuf[buf][k];
    const float dx = P.x - cm.ex, dy = P.y - cm.ey, dz = P.z - cm.ez;
    const float xc = cm.rx * dx + cm.ry * dy + cm.rz * dz;
    const float yc = cm.ux * dx + cm.uy * dy + cm.uz * dz;
    const float zc = cm.fx * dx + cm.fy * dy + cm.fz * dz;
    uint32_t oc = 0;
    oc |= (xc - vw.tl * zc < 0.f) ? 1u : 0u;
    oc |= (vw.tr * zc - xc < 0.f) ? 2u : 0u;
    oc |= (vw.tt * zc - yc < 0.f) ? 4u : 0u;
    oc |= (yc - vw.tb * zc < 0.f) ? 8u : 0u;
    oc |= (zc < cm.near_) ? 16u : 0u;
    ws.vz[k] = zc;
    ws.voc[k] = (uint8_t)oc;
    ws.vfix[k] = zc >= cm.near_ ? project_fix(cm, xc, yc, zc) : make_int2(0, 0);
  }
  __syncwarp();
  for (int tb = 0; tb < nt; tb += 32) {
    const int t = tb + lane;
    bool big = false;
    int npx = 0;
    uint32_t packed = 0;
    if (t < nt) {
      if (kCount) cn.v[kCntTrisSeen]++;
      packed = ws.tbuf[buf][t];
      const int i0 = packed & 0xff, i1 = (packed >> 8) & 0xff, i2 = (packed >> 16) & 0xff;
      const uint32_t oc0 = ws.voc[i0], oc1 = ws.voc[i1], oc2 = ws.voc[i2];
      if ((oc0 & oc1 & oc2) == 0) {
        const float4 P0 = ws.vbuf[buf][i0], P1 = ws.vbuf[buf][i1], P2 = ws.vbuf[buf][i2];
        const float e1x = P1.x - P0.x, e1y = P1.y - P0.y, e1z = P1.z - P0.z;
        const float e2x = P2.x - P0.x, e2y = P2.y - P0.y, e2z = P2.z - P0.z;
        const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z,
                    nz = e1x * e2y - e1y * e2x;
        const float h = nx * (P0.x - cm.ex) + ny * (P0.y - cm.ey) + nz * (P0.z - cm.ez);
        if (h < 0.f) {  // front-facing
          if (kCount) cn.v[kCntTrisFront]++;
          if (((oc0 | oc1 | oc2) & 16u) != 0) {
            big = true;  // crosses the near plane
          } else {
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
              const int ix1 = min(floor_div256(xmax - 128), vw.W - 1);
              const int iy0 = max(ceil_div256(ymin - 128), 0);
              const int iy1 = min(floor_div256(ymax - 128), vw.H - 1);
              if (ix0 <= ix1 && iy0 <= iy1) {
                const int bw = ix1 - ix0 + 1, bh = iy1 - iy0 + 1;
                const bool fits32 = (xmax - xmin) < 32768 && (ymax - ymin) < 32768;
                if (fits32 && bw * bh <= big_px) {
                  // queued for pixel expansion; int32 edge values are exact
                  // because every visited pixel lies inside the bounding box
                  const int2 V[3] = {V0, V1, V2};
                  const int px = ix0 * 256 + 128, py = iy0 * 256 + 128;
                  int e[3], sx[3], sy[3];
#pragma unroll
                  for (int k = 0; k < 3; ++k) {
                    const int dxk = V[(k + 1) % 3].x - V[k].x, dyk = V[(k + 1) % 3].y - V[k].y;
                    e[k] = dxk * (py - V[k].y) - dyk * (px - V[k].x) + (top_left(dxk, dyk) ? 0 : -1);
                    sx[k] = -dyk * 256;
                    sy[k] = dxk * 256;
                  }
                  float A, B, C;
                  depth_plane(cm, nx, ny, nz, h, A, B, C);
                  if (bw <= kDirectW && bh <= kDirectH) {
                    // a box of at most kDirectW x kDirectH pixels (most
                    // triangles of a view) is tested by its own set-up lane:
                    // the same edge values, plane and key as an expansion
                    // slot would compute, without a slot
                    const float u0 = (float)ix0 + 0.5f - cm.cx;
                    const uint32_t rgb = ws.cbuf[buf][t];
#pragma unroll
                    for (int dy = 0; dy < kDirectH; ++dy) {
                      const float row = fmaf(B, (float)(iy0 + dy) + 0.5f - cm.cy, C);
                      unsigned long long* fbp = vw.fb + (iy0 + dy) * vw.W + ix0;
#pragma unroll
                      for (int dx = 0; dx < kDirectW; ++dx)
                        if (dx < bw && dy < bh &&
                            ((e[0] + dx * sx[0] + dy * sy[0]) | (e[1] + dx * sx[1] + dy * sy[1]) |
                             (e[2] + dx * sx[2] + dy * sy[2])) >= 0)
                          frag_key<kCount>(vw, fbp + dx, fmaf(A, u0 + (float)dx, row), rgb, cn);
                    }
                    if (kCount) {
                      cn.v[kCntTrisSmall]++;
                      cn.v[kCntSmallPixels] += bw * bh;
                    }
                  } else {
                    // the record in four 16-byte stores (the round's slot offset follows later)
                    int4* r4 = reinterpret_cast<int4*>(&ws.q[lane]);
                    r4[0] = make_int4(e[0], e[1], e[2], ix0 | (iy0 << 16));
                    r4[1] = make_int4(sx[0], sx[1], sx[2], bw);
                    r4[2] = make_int4(sy[0], sy[1], sy[2], (int)ws.cbuf[buf][t]);
                    r4[3] = make_int4(__float_as_int(A), __float_as_int(B), __float_as_int(C), 0);
                    ws.q[lane].inv_bp = rcp_approx((float)((bw + kSpan - 1) / kSpan));
                    npx = ((bw + kSpan - 1) / kSpan) * bh;  // expansion slots: pixel runs
                    if (kCount) {
                      cn.v[kCntTrisSmall]++;
                      cn.v[kCntSmallPixels] += bw * bh;
                      cn.v[kCntExpandSlots] += npx;
                    }
                  }
                } else {
                  big = true;
                }
              }
            }
          }
        }
      }
    }
    // pixel expansion: the lanes whose triangles have pixels are listed in
    // order (qlane); the c-th listed triangle owns slots [off, off + npx), one
    // slot per pair of horizontally adjacent pixels of its bounding box.  In
    // each pass lane l takes slot base + l (neighbouring lanes mostly take
    // neighbouring pairs of one row); its triangle is the last one started at
    // or before that slot: the ones started in earlier passes plus the start
    // bits of this pass up to lane l.
    int incl = npx;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += v;
    }
    const int off = incl - npx;
    const int total = __shfl_sync(kFull, incl, 31);
    const unsigned has = __ballot_sync(kFull, npx > 0);
    if (npx > 0) {
      ws.q[lane].off = off;
      ws.qlane[__popc(has & ((1u << lane) - 1u))] = (uint8_t)lane;
    }
    if (kCount && lane == 0) {
      cn.v[kCntRounds]++;
      cn.v[kCntExpandTrips] += (total + 31) / 32;
    }
    __syncwarp();
    int started = 0;
    for (int base = 0; base < total; base += 32) {
      const int d = off - base;
      const bool starts = npx > 0 && d >= 0 && d < 32;
      const unsigned smask = __reduce_or_sync(kFull, starts ? (1u << d) : 0u);
      const int k = started + __popc(smask & (0xffffffffu >> (31 - lane))) - 1;
      started += __popc(smask);
      const int s = base + lane;
      if (s < total) {
        // the record in five 16-byte loads: e | ixy, sx | bw, sy | rgb, A B C | off, inv_bp
        const int4* q4 = reinterpret_cast<const int4*>(&ws.q[ws.qlane[k]]);
        const int4 qe = q4[0], qx = q4[1], qy = q4[2], qp = q4[3];
        const float inv_bp = __int_as_float(q4[4].x);
        const int rr = s - qp.w;
        const int bw = qx.w;
        const int y = __float2int_rz(((float)rr + 0.5f) * inv_bp);
        const int x = kSpan * (rr - y * ((bw + kSpan - 1) / kSpan));
        const int e0 = qe.x + x * qx.x + y * qy.x;
        const int e1 = qe.y + x * qx.y + y * qy.y;
        const int e2 = qe.z + x * qx.z + y * qy.z;
        const int i = (qe.w & 0xffff) + x, j = (qe.w >> 16) + y;
        // the run's plane terms once: u + k is exact, so each fragment gets the
        // same value as frag() at (i + k, j)
        const float u0 = (float)i + 0.5f - cm.cx;
        const float row = fmaf(__int_as_float(qp.y), (float)j + 0.5f - cm.cy, __int_as_float(qp.z));
        const float qa = __int_as_float(qp.x);
        unsigned long long* fbp = vw.fb + j * vw.W + i;
#pragma unroll
        for (int u = 0; u < kSpan; ++u)
          if (x + u < bw && ((e0 + u * qx.x) | (e1 + u * qx.y) | (e2 + u * qx.z)) >= 0)
            frag_key<kCount>(vw, fbp + u, fmaf(qa, u0 + (float)u, row), (uint32_t)qy.w, cn);
      }
    }
    __syncwarp();
    unsigned bm = __ballot_sync(kFull, big);
    while (bm) {
      const int L = __ffs(bm) - 1;
      bm &= bm - 1;
      const uint32_t pk = __shfl_sync(kFull, packed, L);
      raster_big<kCount>(vw, cm, ws, buf, pk, ws.cbuf[buf][tb + L], lane, cn);
    }
  }
  __syncwarp();
}

// Offsets and counts of cluster m's vertices and triangles, from its header:
// x = vertex offset | vertex count << 24, y = triangle offset | count << 24.
__device__ __forceinline__ uint2 cluster_entry(const DScene& S, uint32_t m) {
  const float4 h2 = __ldg(S.mhdr + (size_t)kMeshletHdr * m + 2);
  const uint32_t cnt = __float_as_uint(h2.w);
  return make_uint2(__float_as_uint(h2.y) | ((cnt & 0xffu) << 24),
                    __float_as_uint(h2.z) | (((cnt >> 8) & 0xffu) << 24));
}

__device__ __forceinline__ void issue_cluster(WarpSmem& ws, int buf, const DScene& S, uint2 e) {
  const uint32_t voff = e.x & 0xffffffu, nv = e.x >> 24;
  const uint32_t toff = e.y & 0xffffffu, nt = e.y >> 24;
  const uint32_t tbytes = ((nt + 3u) & ~3u) * 4u;
  mbar_expect_tx(&ws.bar[buf], nv * 16u + 2u * tbytes);
  bulk_g2s(ws.vbuf[buf], S.mverts + voff, nv * 16u, &ws.bar[buf]);
  bulk_g2s(ws.tbuf[buf], S.mtris + toff, tbytes, &ws.bar[buf]);
  bulk_g2s(ws.cbuf[buf], S.tri_rgb + toff, tbytes, &ws.bar[buf]);
}

// ---------------------------------------------------------------------------
// Occlusion culling of clusters (two phases per environment).  The depth
// bound of a screen tile of 8x8 pixels is the smallest 1/z over its pixels
// (0 where a pixel is not yet covered), kept as the bits of the positive
// float so that integer order is float order.  Every pixel of the final
// image is at least as near as the bound of its tile, so a cluster whose
// nearest possible point is strictly farther than the bound of every tile
// its screen rectangle touches cannot win any pixel: skipping it leaves the
// image unchanged, bit for bit.
// ---------------------------------------------------------------------------
constexpr int kHizTile = 8;
constexpr float kHizMargin = 1e-4f;  // relative; covers FP32 rounding of both sides

// 1/z bits of a framebuffer key of the current epoch, 0 for background.
__device__ __forceinline__ uint32_t key_invz_bits(unsigned long long key, unsigned long long tag) {
  return (key & (0xffull << 56)) == tag ? ~(uint32_t)(key >> 24) : 0u;
}

// True when the axis-aligned box [lo, hi] (world) lies strictly behind the
// depth bound of every tile its projection touches.  Conservative: a box
// that reaches the near plane, or whose rectangle leaves the image, is kept.
__device__ __forceinline__ bool hiz_occluded(const Cam& cm, const View& vw, float lx, float ly,
                                             float lz, float hx, float hy, float hz,
                                             const uint32_t* hiz) {
  float zmin = CUDART_INF_F, umin = CUDART_INF_F, umax = -CUDART_INF_F, vmin = CUDART_INF_F,
        vmax = -CUDART_INF_F;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float dx = ((k & 1) ? hx : lx) - cm.ex, dy = ((k & 2) ? hy : ly) - cm.ey,
                dz = ((k & 4) ? hz : lz) - cm.ez;
    const float zc = cm.fx * dx + cm.fy * dy + cm.fz * dz;
    const float xc = cm.rx * dx + cm.ry * dy + cm.rz * dz;
    const float yc = cm.ux * dx + cm.uy * dy + cm.uz * dz;
    if (!(zc >= cm.near_)) return false;
    const float iz = 1.f / zc;
    const float u = fmaf(cm.f, xc * iz, cm.cx), v = fmaf(-cm.f, yc * iz, cm.cy);
    zmin = fminf(zmin, zc);
    umin = fminf(umin, u);
    umax = fmaxf(umax, u);
    vmin = fminf(vmin, v);
    vmax = fmaxf(vmax, v);
  }
  // one pixel of slack on every side, then the tiles that rectangle touches
  if (umax < -1.f || vmax < -1.f || umin > (float)vw.W + 1.f || vmin > (float)vw.H + 1.f)
    return false;
  const int tw = vw.W / kHizTile, th = vw.H / kHizTile;
  const int tx0 = max(0, (int)floorf(umin - 1.f) / kHizTile);
  const int tx1 = min(tw - 1, max(0, (int)floorf(umax + 1.f)) / kHizTile);
  const int ty0 = max(0, (int)floorf(vmin - 1.f) / kHizTile);
  const int ty1 = min(th - 1, max(0, (int)floorf(vmax + 1.f)) / kHizTile);
  // the nearest 1/z any point of the box can have, rounded outward
  const uint32_t need = __float_as_uint((1.f / zmin) * (1.f + kHizMargin));
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx)
      if (hiz[ty * tw + tx] <= need) return false;
  return true;
}

// The depth bound of every tile from the framebuffer slot (current epoch).
template <int kW>
__device__ __forceinline__ void hiz_build(const View& vw, uint32_t* hiz, int tid) {
  const int tw = vw.W / kHizTile, tiles = tw * (vw.H / kHizTile);
  for (int t = tid; t < tiles; t += kW * 32) {
    const int tx = t % tw, ty = t / tw;
    uint32_t m = 0xffffffffu;
#pragma unroll 2
    for (int r = 0; r < kHizTile; ++r) {
      const unsigned long long* row = vw.fb + (size_t)(ty * kHizTile + r) * vw.W + tx * kHizTile;
#pragma unroll
      for (int c = 0; c < kHizTile; c += 2) {
        unsigned long long k0, k1;
        asm volatile("ld.global.cg.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
                     : "=l"(k0), "=l"(k1) : "l"(row + c), "l"(vw.pol));
        m = min(m, min(key_invz_bits(k0, vw.tag), key_invz_bits(k1, vw.tag)));
      }
    }
    hiz[t] = m;
  }
}

// Cost class of a visible cluster by the screen radius of its bounding
// sphere (h0: centre, radius): 0 above kClassPx pixels or reaching behind
// the eye, 1 above half that, 2 above a quarter, else 3.  The culled list is
// handed out class by class, costliest first, so that an environment's last
// items are cheap and the warps' wait for one another before the resolve is
// short.
__device__ __forceinline__ uint32_t cluster_class(const Cam& cm, float4 h0) {
  const float zc = cm.fx * (h0.x - cm.ex) + cm.fy * (h0.y - cm.ey) + cm.fz * (h0.z - cm.ez);
  const float rf = h0.w * cm.f;
  return rf > kClassPx * zc ? 0u : rf > 0.5f * kClassPx * zc ? 1u : rf > 0.25f * kClassPx * zc ? 2u : 3u;
}

// The frustum, normal-cone and plane tests of cluster m (as the cull pass
// makes them); its bounding box corners in lo, hi and its cost class when it
// passes.
__device__ __forceinline__ bool cluster_in_view(const DScene& S, int m, const Cam& cm,
                                                const View& vw, float4& lo, float4& hi,
                                                uint32_t& cls) {
  const float4* hd = S.mhdr + (size_t)kMeshletHdr * m;
  const float4 h0 = __ldg(hd);
  if (!sphere_visible(cm, vw, h0.x, h0.y, h0.z, h0.w)) return false;
  cls = cluster_class(cm, h0);
  const float4 h1 = __ldg(hd + 1), h2 = __ldg(hd + 2);
  lo = __ldg(hd + 3);
  hi = __ldg(hd + 4);
  if (h2.x > -0.5f) {
    const float vx = h0.x - cm.ex, vy = h0.y - cm.ey, vz = h0.z - cm.ez;
    const float av = h1.x * vx + h1.y * vy + h1.z * vz;
    const float cx_ = h1.y * vz - h1.z * vy, cy_ = h1.z * vx - h1.x * vz, cz_ = h1.x * vy - h1.y * vx;
    const float cr = sqrtf(cx_ * cx_ + cy_ * cy_ + cz_ * cz_);
    if (av * h2.x - cr * h1.w > h0.w * 1.001f + 1e-4f) return false;
  }
  if (hi.w > 0.5f && h1.x * cm.ex + h1.y * cm.ey + h1.z * cm.ez <
                         lo.w - 1e-4f - 1e-5f * (fabsf(cm.ex) + fabsf(cm.ey) + fabsf(cm.ez)))
    return false;
  return box_visible(cm, vw, lo, hi);
}

__device__ __forceinline__ int pop_item(int* ctr, int lane) {
  int i = 0;
  if (lane == 0) i = atomicAdd(ctr, 1);
  return __shfl_sync(kFull, i, 0);
}

// Per-CTA state of the persistent rasteriser, carried from one environment
// to the next: shared-memory views, the framebuffer slot and its epoch, the
// warp's mbarrier phases and its work counters.
// (The mbarrier phases and the counters, indexed at run time, live in arrays
// of their own beside it, so that the rest stays in registers.)
template <bool kCount>
struct RasterCta {
  int* ctr;         // [0] environment, [2] clusters handed out, [3] objects handed out,
                    // [4..7] clusters listed per cost class, [8..11] their list fill
  uint32_t* list;  // cluster indices of the current pass, in cost-class order
  WarpSmem* ws;
  int tid, lane, warp;
  View vw;
  uint32_t epoch;
  bool dead;        // a wait gave up: this warp stops using its buffers
};

template <bool kCount>
__device__ __forceinline__ void raster_cta_begin(const RasterParams& P, unsigned char* smem,
                                                 RasterCta<kCount>& C, uint32_t phase[2],
                                                 Cnt& cn) {
  C.ctr = reinterpret_cast<int*>(smem);
  C.list = reinterpret_cast<uint32_t*>(smem + 128);
  WarpSmem* wsm = reinterpret_cast<WarpSmem*>(smem + 128 + kListBytes);
  C.tid = threadIdx.x;
  C.lane = C.tid & 31;
  C.warp = C.tid >> 5;
  C.ws = &wsm[C.warp];
  const int npix = P.W * P.H;
  if (kCount)
    for (int k = 0; k < kRasterCounters; ++k) cn.v[k] = 0;
  C.vw.W = P.W;
  C.vw.H = P.H;
  C.vw.fb = P.fb_slots + (size_t)blockIdx.x * npix;
  C.epoch = P.fb_epoch ? P.fb_epoch[blockIdx.x] : 0u;  // slot epochs persist across launches
  // the slot stays in L2 while observations stream through it
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(C.vw.pol));
  if (C.lane == 0) {
    mbar_init(&C.ws->bar[0]);
    mbar_init(&C.ws->bar[1]);
    fence_mbar_init();
  }
  phase[0] = phase[1] = 0u;
  C.dead = false;
}

// Renders environment env into its observation rows (the whole CTA of kW
// warps).  kBoxes: the objects are oriented boxes (P.obox), drawn as cubes;
// a separate instantiation, so the sphere objects' code stays as it is.
// kOcc: clusters are culled by occlusion in two phases -- first the clusters
// this environment showed in its previous image (visibility bits P.vis),
// then the depth bound of every 8x8 tile is taken from the framebuffer and
// the other clusters (and the objects) are drawn only when some tile they
// touch could still show them; after the resolve the bits are rewritten from
// the final image's tile bounds.  The image is the same bit for bit.
template <bool kCount, int kW, bool kBoxes = false, bool kOcc = false>
__device__ __forceinline__ void render_env(const RasterParams& P, const int env,
                                           RasterCta<kCount>& C, uint32_t phase[2], Cnt& cn) {
  int* ctr = C.ctr;
  uint32_t* list = C.list;
  WarpSmem& ws = *C.ws;
  const int tid = C.tid, lane = C.lane;
  View& vw = C.vw;
  uint32_t& epoch = C.epoch;
  bool& dead = C.dead;
  const int W = P.W, H = P.H, npix = W * H;
  (void)W;
  (void)H;
  // a new epoch for this slot: its keys outrank every older key, so the slot
  // needs no clearing between environments; every 255 environments it wraps
  // and is cleared once
  if (++epoch == 256u) {
    for (int p = tid * 2; p < npix; p += kW * 32 * 2)
      asm volatile("st.global.cg.L2::cache_hint.v2.u64 [%0], {%1, %1}, %2;" ::"l"(vw.fb + p),
                   "l"(~0ull), "l"(vw.pol)
                   : "memory");
    __threadfence();
    __syncthreads();
    epoch = 1u;
  }
  vw.tag = (unsigned long long)(255u - epoch) << 56;
  // a scene index outside the set is refused before any scene data is
  // read: the environment is drawn empty (no clusters, no objects), so its
  // images resolve to background, and an error bit is set
  const int scene = P.env_scene[env];
  const bool scene_ok = (unsigned)scene < (unsigned)P.n_scenes;
  if (!scene_ok && tid == 0) atomicOr(P.err, kErrBadScene);
  const DScene& S = P.scenes[scene_ok ? scene : 0];
  Cam cm;
  {
    const float* c = P.cam + (size_t)env * 12;
    cm.rx = c[0]; cm.ux = c[1]; cm.fx = c[2];
    cm.ry = c[3]; cm.uy = c[4]; cm.fy = c[5];
    cm.rz = c[6]; cm.uz = c[7]; cm.fz = c[8];
    cm.ex = c[9]; cm.ey = c[10]; cm.ez = c[11];
    cm.f = 0.5f * (float)W;
    cm.cx = 0.5f * (float)W;
    cm.cy = 0.5f * (float)H;
    cm.near_ = P.near_;
  }
  vw.tl = (-1.f - cm.cx) / cm.f;
  vw.tr = ((float)W + 1.f - cm.cx) / cm.f;
  vw.tt = (cm.cy + 1.f) / cm.f;
  vw.tb = (cm.cy - ((float)H + 1.f)) / cm.f;
  vw.kl = rsqrtf(1.f + vw.tl * vw.tl);
  vw.kr = rsqrtf(1.f + vw.tr * vw.tr);
  vw.kt = rsqrtf(1.f + vw.tt * vw.tt);
  vw.kb = rsqrtf(1.f + vw.tb * vw.tb);

  // occlusion culling: tile depth bounds after the bytes of the warps' buffers;
  // the environment's visibility bits (one per cluster)
  uint32_t* hiz = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(ctr) + 128 +
                                              kListBytes + kW * sizeof(WarpSmem));
  uint32_t* visw = kOcc ? P.vis + (size_t)env * P.vis_words : nullptr;
  constexpr int kPhases = kOcc ? 2 : 1;
#pragma unroll 1
  for (int ph = 0; ph < kPhases; ++ph) {
  for (int base = 0; scene_ok && (base < S.n_meshlets || base == 0); base += kListCap) {
    if (tid >= 1 && tid < 12) ctr[tid] = 0;
    __syncthreads();
    // 1. the whole CTA culls the clusters of this pass; a visible one gets a
    //    3-bit code per loop trip (1 + its cost class) and is counted in its class
    const int end = min(base + kListCap, S.n_meshlets);
    // 3 bits per trip: a 32-bit word holds 10 trips, more need 64 bits
    constexpr int kTrips = (kListCap + kW * 32 - 1) / (kW * 32);
    static_assert(kTrips <= 21, "codes of one pass in 63 bits");
    using Codes = typename std::conditional<(kTrips > 10), unsigned long long, uint32_t>::type;
    Codes codes = 0;
    int trip = 0;
    if (kOcc) {
      for (int m = base + tid; m < end; m += kW * 32, ++trip) {
        if (kCount && ph == 0) cn.v[kCntClustersTested]++;
        const bool prev = (visw[m >> 5] >> (m & 31)) & 1u;
        if (ph == 0 && !prev) continue;
        if (ph == 1 && prev) continue;  // drawn in the first phase
        float4 lo, hi;
        uint32_t cls;
        if (!cluster_in_view(S, m, cm, vw, lo, hi, cls)) continue;
        if (ph == 1 && hiz_occluded(cm, vw, lo.x, lo.y, lo.z, hi.x, hi.y, hi.z, hiz)) {
          if (kCount) cn.v[kCntClustersOccluded]++;
          continue;
        }
        codes |= (Codes)(1u + cls) << (3 * trip);
        atomicAdd(&ctr[4 + cls], 1);
      }
    } else
    for (int m = base + tid; m < end; m += kW * 32, ++trip) {
      if (kCount) cn.v[kCntClustersTested]++;
      const float4* hd = S.mhdr + (size_t)kMeshletHdr * m;
      const float4 h0 = __ldg(hd);
      bool vis = sphere_visible(cm, vw, h0.x, h0.y, h0.z, h0.w);
      if (vis) {
        const float4 h1 = __ldg(hd + 1), h2 = __ldg(hd + 2), h3 = __ldg(hd + 3),
                     h4 = __ldg(hd + 4);
        if (h2.x > -0.5f) {  // normal cone: every face looks away from the eye
          const float vx = h0.x - cm.ex, vy = h0.y - cm.ey, vz = h0.z - cm.ez;
          const float av = h1.x * vx + h1.y * vy + h1.z * vz;
          const float cx_ = h1.y * vz - h1.z * vy, cy_ = h1.z * vx - h1.x * vz,
                      cz_ = h1.x * vy - h1.y * vx;
          const float cr = sqrtf(cx_ * cx_ + cy_ * cy_ + cz_ * cz_);
          if (av * h2.x - cr * h1.w > h0.w * 1.001f + 1e-4f) vis = false;
        }
        // one face normal: back-facing as a whole when the eye is on the back
        // side of (or on) every face's plane
        if (vis && h4.w > 0.5f &&
            h1.x * cm.ex + h1.y * cm.ey + h1.z * cm.ez <
                h3.w - 1e-4f - 1e-5f * (fabsf(cm.ex) + fabsf(cm.ey) + fabsf(cm.ez)))
          vis = false;
        if (vis) vis = box_visible(cm, vw, h3, h4);
        if (vis) {
          const uint32_t cls = cluster_class(cm, h0);
          codes |= (Codes)(1u + cls) << (3 * trip);
          atomicAdd(&ctr[4 + cls], 1);
        }
      }
    }
    __syncthreads();
    // 2. the list in class order (a counting sort): each thread places the
    //    indices of its visible clusters
    for (int m = base + tid, t = 0; (codes >> (3 * t)) != 0u; m += kW * 32, ++t) {
      const uint32_t code = (uint32_t)(codes >> (3 * t)) & 7u;
      if (code == 0u) continue;
      const int at = (code > 1u ? ctr[4] : 0) + (code > 2u ? ctr[5] : 0) +
                     (code > 3u ? ctr[6] : 0) + atomicAdd(&ctr[7 + code], 1);
      list[at] = (uint32_t)m;
    }
    __syncthreads();
    const int count = ctr[4] + ctr[5] + ctr[6] + ctr[7];
    // 3. warps take one cluster at a time; the next streams in meanwhile
    int cur = dead ? count : pop_item(&ctr[2], lane);
    int buf = 0;
    if (cur < count && lane == 0) {
      ws.ent[0] = cluster_entry(S, list[cur]);
      issue_cluster(ws, 0, S, ws.ent[0]);
    }
    __syncwarp();
    while (cur < count) {
      const int nxt = pop_item(&ctr[2], lane);
      if (nxt < count && lane == 0) {
        // the other buffer's entry is free: its cluster was drawn, and the
        // draw ended with a warp synchronisation
        ws.ent[buf ^ 1] = cluster_entry(S, list[nxt]);
        issue_cluster(ws, buf ^ 1, S, ws.ent[buf ^ 1]);
      }
      const bool ok = mbar_wait(&ws.bar[buf], phase[buf],
                                (kCount && lane == 0) ? &cn.v[kCntWaitIters] : nullptr);
      phase[buf] ^= 1u;
      if (!__all_sync(kFull, ok)) {
        if (lane == 0) atomicOr(P.err, kErrWaitTimeout);
        // let the copy in flight into the other buffer land before leaving
        if (nxt < count) mbar_wait(&ws.bar[buf ^ 1], phase[buf ^ 1]);
        dead = true;
        break;
      }
      const uint2 e = ws.ent[buf];
      raster_cluster<kCount>(vw, cm, ws, buf, (int)(e.x >> 24), (int)(e.y >> 24), P.big_px,
                             lane, cn);
      cur = nxt;
      buf ^= 1;
    }
    // 4. free objects (last pass): icosahedra scaled to each object's radius
    if (ph == kPhases - 1 && base + kListCap >= S.n_meshlets) {
      // objects, then (when rendered) the robot's 32 sphere slots, which
      // take instance slots 64.. so their colours follow the objects'
      const int n_inst = P.M + (P.robot_sph ? 32 : 0);
      while (!dead) {
        const int j = pop_item(&ctr[3], lane);
        if (j >= n_inst) break;
        const float4 o = j < P.M ? P.obj[(size_t)env * P.M + j]
                                 : P.robot_sph[(size_t)env * 32 + (j - P.M)];
        if (!(o.w > 0.f)) continue;
        const int slot = j < P.M ? j : GX_MAX_OBJECTS + (j - P.M);
        if (!sphere_visible(cm, vw, o.x, o.y, o.z, o.w * 1.0001f + 1e-6f)) continue;
        if (kOcc) {
          const float r = o.w * 1.0001f + 1e-6f;
          if (hiz_occluded(cm, vw, o.x - r, o.y - r, o.z - r, o.x + r, o.y + r, o.z + r, hiz))
            continue;
        }
        const uint32_t rgb = __ldg(P.obj_rgb + slot);
        int nv = P.omesh_nv, nt = P.omesh_nt;
        if (kBoxes) {
          // an oriented box (its bounding sphere was culled above): the unit
          // cube, corner k = signs of bits 0/1/2 of k, mapped by its world
          // rotation times diag(half extents) -- R_y(yaw) resting, the
          // tool-carried rotation while held
          float4 r0, r1, r2;
          if (j == P.held[env]) {
            r0 = P.held_M[(size_t)env * 3];
            r1 = P.held_M[(size_t)env * 3 + 1];
            r2 = P.held_M[(size_t)env * 3 + 2];
          } else {
            const float4 b = P.obox[(size_t)env * P.M + j];
            float sy, cy;
            sincosf(b.w, &sy, &cy);
            r0 = make_float4(cy * b.x, 0.f, sy * b.z, 0.f);
            r1 = make_float4(0.f, b.y, 0.f, 0.f);
            r2 = make_float4(-sy * b.x, 0.f, cy * b.z, 0.f);
          }
          if (lane < 8) {
            const float ux = (lane & 1) ? 1.f : -1.f, uy = (lane & 2) ? 1.f : -1.f,
                        uz = (lane & 4) ? 1.f : -1.f;
            ws.vbuf[0][lane] = make_float4(fmaf(r0.x, ux, fmaf(r0.y, uy, fmaf(r0.z, uz, o.x))),
                                           fmaf(r1.x, ux, fmaf(r1.y, uy, fmaf(r1.z, uz, o.y))),
                                           fmaf(r2.x, ux, fmaf(r2.y, uy, fmaf(r2.z, uz, o.z))),
                                           0.f);
          }
          if (lane < 12) {
            ws.tbuf[0][lane] = kCubeTris[lane];
            ws.cbuf[0][lane] = rgb;
          }
          nv = 8;
          nt = 12;
        } else {
          for (int k = lane; k < P.omesh_nv; k += 32) {
            const float4 u = P.omesh_v[k];
            ws.vbuf[0][k] = make_float4(fmaf(o.w, u.x, o.x), fmaf(o.w, u.y, o.y),
                                        fmaf(o.w, u.z, o.z), 0.f);
          }
          for (int k = lane; k < P.omesh_nt; k += 32) {
            ws.tbuf[0][k] = P.omesh_t[k];
            ws.cbuf[0][k] = rgb;
          }
        }
        __syncwarp();
        raster_cluster<kCount>(vw, cm, ws, 0, nv, nt, P.big_px, lane, cn);
      }
      // object vertices were written to vbuf[0] by ordinary stores: order
      // them before later bulk copies into the same buffer
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();  // the list is reused by the next pass
  }
  if (kOcc && ph == 0) {
    // the first phase's fragments must land before their tile bounds are read
    __threadfence();
    __syncthreads();
    hiz_build<kW>(vw, hiz, tid);
    __syncthreads();
  }
  }
  if (kOcc) {  // the final image's tile bounds are gathered during the resolve
    const int tiles = (W / kHizTile) * (H / kHizTile);
    for (int t = tid; t < tiles; t += kW * 32) hiz[t] = 0xffffffffu;
  }
  // the reductions must land before the resolve reads the slot
  __threadfence();
  __syncthreads();

  // resolve four pixels per thread: 16-byte streaming stores, row-major; the
  // slot is read from L2 and left as it is (the next environment's keys carry
  // a newer epoch); keys of older epochs are background
  const size_t out0 = (size_t)env * npix;
  for (int p = tid * 4; p < npix; p += kW * 32 * 4) {
    unsigned long long keys[4];
    asm volatile("ld.global.cg.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
                 : "=l"(keys[0]), "=l"(keys[1]) : "l"(vw.fb + p), "l"(vw.pol));
    asm volatile("ld.global.cg.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
                 : "=l"(keys[2]), "=l"(keys[3]) : "l"(vw.fb + p + 2), "l"(vw.pol));

    float z[4];
    uint32_t col[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      z[k] = 0.f;
      col[k] = 0u;
      if ((keys[k] & (0xffull << 56)) == vw.tag) {  // written in this epoch
        const float invz = __uint_as_float(~(uint32_t)(keys[k] >> 24));
        z[k] = rcp_approx(invz);
        col[k] = (uint32_t)keys[k] & 0xffffffu;  // the winner's colour rides in the key
      }
    }
    if (kOcc) {
      const uint32_t b = min(min(key_invz_bits(keys[0], vw.tag), key_invz_bits(keys[1], vw.tag)),
                             min(key_invz_bits(keys[2], vw.tag), key_invz_bits(keys[3], vw.tag)));
      const int row = p / W, col0 = p - row * W;
      atomicMin(&hiz[(row / kHizTile) * (W / kHizTile) + col0 / kHizTile], b);
    }
    if (P.depth_fp16) {
      __half2 a = __floats2half2_rn(z[0], z[1]), b = __floats2half2_rn(z[2], z[3]);
      uint2 v;
      v.x = *reinterpret_cast<uint32_t*>(&a);
      v.y = *reinterpret_cast<uint32_t*>(&b);
      __stcs(reinterpret_cast<uint2*>(reinterpret_cast<__half*>(P.depth) + out0 + p), v);
    } else {
      __stcs(reinterpret_cast<float4*>(reinterpret_cast<float*>(P.depth) + out0 + p),
             make_float4(z[0], z[1], z[2], z[3]));
    }
    if (P.rgb) {
      // 4 pixels = 12 bytes R G B R G B ... packed into three words
      // (one byte permutation per word: colours are 0x00RRGGBB)
      const uint32_t r0 = col[0], r1 = col[1], r2 = col[2], r3 = col[3];
      const uint32_t w0 = __byte_perm(r0, r1, 0x6012);  // R0 G0 B0 R1
      const uint32_t w1 = __byte_perm(r1, r2, 0x5601);  // G1 B1 R2 G2
      const uint32_t w2 = __byte_perm(r2, r3, 0x4560);  // B2 R3 G3 B3
      unsigned int* o = reinterpret_cast<unsigned int*>(P.rgb + (out0 + p) * 3);
      __stcs(o, w0);
      __stcs(o + 1, w1);
      __stcs(o + 2, w2);
    }
  }
  __syncthreads();
  if (kOcc && scene_ok) {
    // next image's first phase: the clusters in view that the final image's
    // tile bounds do not rule out, one bit per cluster, a ballot per word
    const int warp = C.warp;
    for (int m0 = warp * 32; m0 < S.n_meshlets; m0 += kW * 32) {
      const int m = m0 + lane;
      bool v = false;
      if (m < S.n_meshlets) {
        float4 lo, hi;
        uint32_t cls;
        v = cluster_in_view(S, m, cm, vw, lo, hi, cls) &&
            !hiz_occluded(cm, vw, lo.x, lo.y, lo.z, hi.x, hi.y, hi.z, hiz);
      }
      const unsigned b = __ballot_sync(kFull, v);
      if (lane == 0) visw[m0 >> 5] = b;
    }
    __syncthreads();
  }
}

// Writes back the slot's epoch and the work counters.
template <bool kCount>
__device__ __forceinline__ void raster_cta_end(const RasterParams& P, RasterCta<kCount>& C,
                                               Cnt& cn) {
  const int tid = C.tid, lane = C.lane;
  const uint32_t epoch = C.epoch;
  if (P.fb_epoch && tid == 0) P.fb_epoch[blockIdx.x] = epoch;
  if (kCount) {
    for (int k = 0; k < kRasterCounters; ++k) {
      unsigned long long v = cn.v[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
      if (lane == 0 && v) atomicAdd(P.counters + k, v);
    }
  }
}

}  // namespace rast
}  // namespace
}  // namespace gx
