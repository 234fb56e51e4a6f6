// Device functions shared by the step kernels and the neural-SDF kernels:
// the counter-based random generator and the distance-grid query.
#pragma once

#include <math_constants.h>

#include "gx_internal.h"

// Where this translation unit's kernels read distance-grid nodes: 0 the dense
// grid only, 1 the box store only (a second instantiation of the step
// kernels), 2 chosen per scene at run time by DScene::store (set-up and query
// kernels).  The step kernels are compiled once per store so the dense path
// keeps its register allocation.
#ifndef GX_STATIC_STORE
#define GX_STATIC_STORE 0
#endif

namespace gx {
namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor S-box with a Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ float unit24(uint32_t w) {
  return (float)(w >> 8) * (1.0f / 16777216.0f);
}

#if GX_STATIC_STORE == 1
#define GX_STORE_INLINE __forceinline__
#else
#define GX_STORE_INLINE __noinline__
#endif

// Box store (DScene::store == 1): a node's value is recomputed from the
// scene's solid boxes instead of read from the dense grid.  The lattice is
// cut into cells of 16 node intervals per axis; cell c lists the boxes that
// can be nearest anywhere in its nodes [16c, 16c + 16] (a superset of the
// argmin, chosen on the host by exact convex bounds), so the minimum over the
// list equals the minimum over all boxes.  FP32: within ~1e-5 m of the FP64
// node value for coordinates up to ~20 m.
__device__ __forceinline__ const uint16_t* store_list(const DScene& s, int i, int j, int k,
                                                      int& n) {
  const int ci = min(i >> kStoreShift, s.sbx - 1), cj = min(j >> kStoreShift, s.sby - 1),
            ck = min(k >> kStoreShift, s.sbz - 1);
  const int c = (ck * s.sby + cj) * s.sbx + ci;
  const uint32_t a = __ldg(s.sb_off + c), b = __ldg(s.sb_off + c + 1);
  n = (int)(b - a);
  return s.sb_ids + a;
}

// Signed distance of the union of boxes at node (i, j, k): for each box the
// per-axis excess q = |p - centre| - half; outside (max q > 0) the distance
// is |max(q, 0)|, inside it is max q.  min over boxes of both parts at once:
// out2 = min of |max(q, 0)|^2 (0 when some box holds p) and in = min(0, min
// of max q), so the value is sqrt(out2) + in.
__device__ GX_STORE_INLINE float store_node(const DScene& s, int i, int j, int k) {
  int n;
  const uint16_t* ids = store_list(s, i, j, k, n);
  const float x = fmaf((float)i, s.h, s.ox), y = fmaf((float)j, s.h, s.oy),
              z = fmaf((float)k, s.h, s.oz);
  float out2 = CUDART_INF_F, in = 0.f;
  for (int t = 0; t < n; ++t) {
    const int b = __ldg(ids + t);
    const float4 c = __ldg(s.sbox + 2 * b), e = __ldg(s.sbox + 2 * b + 1);
    const float qx = fabsf(x - c.x) - e.x, qy = fabsf(y - c.y) - e.y, qz = fabsf(z - c.z) - e.z;
    const float px = fmaxf(qx, 0.f), py = fmaxf(qy, 0.f), pz = fmaxf(qz, 0.f);
    out2 = fminf(out2, __fadd_rn(__fadd_rn(__fmul_rn(px, px), __fmul_rn(py, py)), __fmul_rn(pz, pz)));
    in = fminf(in, fmaxf(qx, fmaxf(qy, qz)));
  }
  return sqrtf(out2) + in;
}

// The eight corners of lattice cell (i, j, k) from the box store, one list.
__device__ GX_STORE_INLINE void store_cell(const DScene& s, int i, int j, int k, float cc[8]) {
  int n;
  const uint16_t* ids = store_list(s, i, j, k, n);
  const float x0 = fmaf((float)i, s.h, s.ox), x1 = fmaf((float)(i + 1), s.h, s.ox);
  const float y0 = fmaf((float)j, s.h, s.oy), y1 = fmaf((float)(j + 1), s.h, s.oy);
  const float z0 = fmaf((float)k, s.h, s.oz), z1 = fmaf((float)(k + 1), s.h, s.oz);
  float out2[8], in[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    out2[v] = CUDART_INF_F;
    in[v] = 0.f;
  }
  for (int t = 0; t < n; ++t) {
    const int b = __ldg(ids + t);
    const float4 c = __ldg(s.sbox + 2 * b), e = __ldg(s.sbox + 2 * b + 1);
    const float qx[2] = {fabsf(x0 - c.x) - e.x, fabsf(x1 - c.x) - e.x};
    const float qy[2] = {fabsf(y0 - c.y) - e.y, fabsf(y1 - c.y) - e.y};
    const float qz[2] = {fabsf(z0 - c.z) - e.z, fabsf(z1 - c.z) - e.z};
    float sx[2], sy[2], sz[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const float px = fmaxf(qx[a], 0.f), py = fmaxf(qy[a], 0.f), pz = fmaxf(qz[a], 0.f);
      sx[a] = __fmul_rn(px, px);  // no contraction: store_node rounds the same way
      sy[a] = __fmul_rn(py, py);
      sz[a] = __fmul_rn(pz, pz);
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {  // corner v: x offset bit 0, y bit 1, z bit 2
      const int a = v & 1, bb = (v >> 1) & 1, cz = v >> 2;
      out2[v] = fminf(out2[v], __fadd_rn(__fadd_rn(sx[a], sy[bb]), sz[cz]));
      in[v] = fminf(in[v], fmaxf(qx[a], fmaxf(qy[bb], qz[cz])));
    }
  }
#pragma unroll
  for (int v = 0; v < 8; ++v) cc[v] = sqrtf(out2[v]) + in[v];
}

__device__ __forceinline__ float gnode(const DScene& s, int i, int j, int k) {
#if GX_STATIC_STORE == 1
  return store_node(s, i, j, k);
#else
#if GX_STATIC_STORE == 2
  if (s.store) return store_node(s, i, j, k);
#endif
  return __ldg(s.grid + ((size_t)k * s.ny + j) * s.nx + i);
#endif
}

// Corner values of lattice cell (i, j, k), corner v at (i + (v & 1),
// j + (v >> 1 & 1), k + (v >> 2)), from the dense grid or the box store.
__device__ __forceinline__ void cell_corners(const DScene& s, int i, int j, int k, float cc[8]) {
#if GX_STATIC_STORE == 1
  store_cell(s, i, j, k, cc);
  return;
#endif
#if GX_STATIC_STORE == 2
  if (s.store) {
    store_cell(s, i, j, k, cc);
    return;
  }
#endif
  const float* g = s.grid + ((size_t)k * s.ny + j) * s.nx + i;
  const size_t sy = s.nx, sz = (size_t)s.nx * s.ny;
  cc[0] = __ldg(g);
  cc[1] = __ldg(g + 1);
  cc[2] = __ldg(g + sy);
  cc[3] = __ldg(g + sy + 1);
  cc[4] = __ldg(g + sz);
  cc[5] = __ldg(g + sz + 1);
  cc[6] = __ldg(g + sz + sy);
  cc[7] = __ldg(g + sz + sy + 1);
}

__device__ __forceinline__ float lerp8(const float cc[8], float tx, float ty, float tz) {
  const float c00 = cc[0] + tx * (cc[1] - cc[0]), c10 = cc[2] + tx * (cc[3] - cc[2]);
  const float c01 = cc[4] + tx * (cc[5] - cc[4]), c11 = cc[6] + tx * (cc[7] - cc[6]);
  const float c0 = c00 + ty * (c10 - c00), c1 = c01 + ty * (c11 - c01);
  return c0 + tz * (c1 - c0);
}

// Trilinear interpolation at lattice coordinates g (0 <= g <= n - 1 per axis).
__device__ __forceinline__ float grid_lerp(const DScene& s, float gx, float gy, float gz) {
  const int i = min((int)floorf(gx), s.nx - 2);
  const int j = min((int)floorf(gy), s.ny - 2);
  const int k = min((int)floorf(gz), s.nz - 2);
  const float tx = gx - i, ty = gy - j, tz = gz - k;
  float cc[8];
  cell_corners(s, i, j, k, cc);
  return lerp8(cc, tx, ty, tz);
}

// Trilinear distance and its horizontal gradient (x and z, per metre) at c;
// false outside the lattice box.  d equals grid_query's value.
__device__ bool grid_query_grad(const DScene& s, float cx, float cy, float cz, float& d,
                                float& gxo, float& gzo) {
  const float gx = (cx - s.ox) * s.inv_h, gy = (cy - s.oy) * s.inv_h, gz = (cz - s.oz) * s.inv_h;
  if (!(gx >= 0.f && gx <= (float)(s.nx - 1) && gy >= 0.f && gy <= (float)(s.ny - 1) &&
        gz >= 0.f && gz <= (float)(s.nz - 1)))
    return false;
  const int i = min((int)floorf(gx), s.nx - 2);
  const int j = min((int)floorf(gy), s.ny - 2);
  const int k = min((int)floorf(gz), s.nz - 2);
  const float tx = gx - i, ty = gy - j, tz = gz - k;
  float cc[8];
  cell_corners(s, i, j, k, cc);
  d = lerp8(cc, tx, ty, tz);
  const float c000 = cc[0], c100 = cc[1], c010 = cc[2], c110 = cc[3];
  const float c001 = cc[4], c101 = cc[5], c011 = cc[6], c111 = cc[7];
  gxo = ((c100 - c000) * (1.f - ty) * (1.f - tz) + (c110 - c010) * ty * (1.f - tz) +
         (c101 - c001) * (1.f - ty) * tz + (c111 - c011) * ty * tz) * s.inv_h;
  gzo = ((c001 - c000) * (1.f - tx) * (1.f - ty) + (c101 - c100) * tx * (1.f - ty) +
         (c011 - c010) * (1.f - tx) * ty + (c111 - c110) * tx * ty) * s.inv_h;
  return true;
}

// Column-grid test of a sphere (c, r): the smallest working-set radius R not
// below r (1e-5 relative tolerance), the nearest column (floor(f + 0.5)),
// contact unless the centre height lies in one of the column's free spans
// widened by R - r at both ends; outside the columns' extent is contact.
__device__ bool column_contact(const DScene& s, float cx, float cy, float cz, float r) {
  const int ri = r <= 0.015f * 1.00001f ? 0 : (r <= 0.05f * 1.00001f ? 1 : 2);
  // spans are for radius R >= r: widened by R - r at both ends
  const float w = fmaxf((ri == 0 ? 0.015f : (ri == 1 ? 0.05f : 0.12f)) - r, 0.f);
  const float fi = (cx - s.ox) * (float)(1.0 / kColumnSpacing);
  const float fk = (cz - s.oz) * (float)(1.0 / kColumnSpacing);
  if (!(fi > -0.5f && fk > -0.5f)) return true;  // also catches NaN
  const int i = (int)floorf(fi + 0.5f), k = (int)floorf(fk + 0.5f);
  if (i >= s.ncx || k >= s.ncz) return true;
  const int idx = (ri * s.ncz + k) * s.ncx + i;
  const uint32_t a = __ldg(s.col_off + idx), b = __ldg(s.col_off + idx + 1);
  for (uint32_t t = a; t < b; ++t) {
    const float2 sp = __ldg(s.col_spans + t);
    if (cy >= sp.x - w && cy <= sp.y + w) return false;
  }
  return true;
}

// Broad-phase cell range of an object (x, z, radius rho) in grid g, padded
// by 0.1 mm so rounding can only add cells; false outside the lattice.
__device__ __forceinline__ void bp_range(const DScene& s, int g, float x, float z, float rho,
                                         int& i0, int& i1, int& k0, int& k1) {
  const float sx = (g & 1) ? 0.5f * kBpCell : 0.f, sz = (g & 2) ? 0.5f * kBpCell : 0.f;
  const float inv = 1.f / kBpCell, pad = rho + 1e-4f;
  i0 = max((int)floorf((x - pad - s.bp_x0 - sx) * inv), 0);
  i1 = min((int)floorf((x + pad - s.bp_x0 - sx) * inv), s.bp_nx - 1);
  k0 = max((int)floorf((z - pad - s.bp_z0 - sz) * inv), 0);
  k1 = min((int)floorf((z + pad - s.bp_z0 - sz) * inv), s.bp_nz - 1);
}
__device__ __forceinline__ void bp_insert(BpCell* grids, int cells, const DScene& s, int j,
                                          float x, float z, float rho) {
  for (int g = 0; g < 4; ++g) {
    int i0, i1, k0, k1;
    bp_range(s, g, x, z, rho, i0, i1, k0, k1);
    for (int k = k0; k <= k1; ++k)
      for (int i = i0; i <= i1; ++i) {
        BpCell& c = grids[(size_t)g * cells + (size_t)k * s.bp_nx + i];
        const uint32_t slot = atomicAdd(&c.count, 1u);
        if (slot < (uint32_t)kBpCap) c.id[slot] = (uint8_t)j;
      }
  }
}
// Removes object j from its cells (single thread per environment); a cell
// that ever overflowed stays in brute-force mode until the next rebuild.
__device__ __forceinline__ void bp_remove(BpCell* grids, int cells, const DScene& s, int j,
                                          float x, float z, float rho) {
  for (int g = 0; g < 4; ++g) {
    int i0, i1, k0, k1;
    bp_range(s, g, x, z, rho, i0, i1, k0, k1);
    for (int k = k0; k <= k1; ++k)
      for (int i = i0; i <= i1; ++i) {
        BpCell& c = grids[(size_t)g * cells + (size_t)k * s.bp_nx + i];
        if (c.count > (uint32_t)kBpCap) continue;
        for (uint32_t t = 0; t < c.count; ++t)
          if (c.id[t] == (uint8_t)j) {
            c.id[t] = c.id[c.count - 1];
            c.count -= 1;
            break;
          }
      }
  }
}
// The cell of the grid that holds the whole XZ disk of a query sphere;
// nullptr when there is none in range (the caller tests every object).
__device__ __forceinline__ const BpCell* bp_cell(const BpCell* grids, int cells, const DScene& s,
                                                 float x, float z, float r) {
  const float inv = 1.f / kBpCell, h = 0.5f * kBpCell;
  int g = 0, ci = 0, ck = 0;
  {
    const float a = (x - s.bp_x0) * inv;
    const int lo = (int)floorf(a - r * inv), hi = (int)floorf(a + r * inv);
    if (lo == hi) {
      ci = lo;
    } else {
      g |= 1;
      ci = (int)floorf((x - r - s.bp_x0 - h) * inv);
      if ((int)floorf((x + r - s.bp_x0 - h) * inv) != ci) return nullptr;
    }
  }
  {
    const float a = (z - s.bp_z0) * inv;
    const int lo = (int)floorf(a - r * inv), hi = (int)floorf(a + r * inv);
    if (lo == hi) {
      ck = lo;
    } else {
      g |= 2;
      ck = (int)floorf((z - r - s.bp_z0 - h) * inv);
      if ((int)floorf((z + r - s.bp_z0 - h) * inv) != ck) return nullptr;
    }
  }
  if (ci < 0 || ci >= s.bp_nx || ck < 0 || ck >= s.bp_nz) return nullptr;
  const BpCell* c = grids + (size_t)g * cells + (size_t)ck * s.bp_nx + ci;
  return c->count > (uint32_t)kBpCap ? nullptr : c;
}

// true when c lies inside the lattice box (and is finite).
__device__ __forceinline__ bool grid_contains(const DScene& s, float cx, float cy, float cz) {
  const float gx = (cx - s.ox) * s.inv_h, gy = (cy - s.oy) * s.inv_h, gz = (cz - s.oz) * s.inv_h;
  return gx >= 0.f && gx <= (float)(s.nx - 1) && gy >= 0.f && gy <= (float)(s.ny - 1) &&
         gz >= 0.f && gz <= (float)(s.nz - 1);
}

// Trilinear interpolation of the distance grid.  false when c lies outside
// the lattice box (or is not finite): that counts as contact.
__device__ bool grid_query(const DScene& s, float cx, float cy, float cz, float& d) {
  const float gx = (cx - s.ox) * s.inv_h, gy = (cy - s.oy) * s.inv_h, gz = (cz - s.oz) * s.inv_h;
  if (!(gx >= 0.f && gx <= (float)(s.nx - 1) && gy >= 0.f && gy <= (float)(s.ny - 1) &&
        gz >= 0.f && gz <= (float)(s.nz - 1)))
    return false;
  d = grid_lerp(s, gx, gy, gz);
  return true;
}

// Fourier-feature phase b . (p - c) in turns, reduced to about [-1/2, 1/2].
// FP32 alone loses the phase of a point metres from c (|b . (p - c)| reaches
// tens of turns, ~1e-5 rad of rounding); the difference p - c (Knuth's
// TwoSum) and the products (FMA TwoProduct) are carried as unevaluated
// hi + lo pairs, the integer part of hi is removed exactly, and only the
// final fraction is rounded, so the phase is good to ~1e-7 rad.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
struct Centred {
  float h[3], l[3];
};
__device__ __forceinline__ Centred centre_point(float x, float y, float z, const float c[3]) {
  Centred d;
  two_sum(x, -c[0], d.h[0], d.l[0]);
  two_sum(y, -c[1], d.h[1], d.l[1]);
  two_sum(z, -c[2], d.h[2], d.l[2]);
  return d;
}
// sin and cos of 2 pi t for a reduced phase t (|t| <= ~1/2): the hardware
// approximations, absolute error below 4e-7 on [-pi, pi].
__device__ __forceinline__ void sincos_turns(float t, float* s, float* c) {
  const float a = 6.2831853071795865f * t;
  *s = __sinf(a);
  *c = __cosf(a);
}

__device__ __forceinline__ float phase_turns(const float b[3], const Centred& d) {
  float hi = 0.f, lo = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float p = b[a] * d.h[a];
    const float pe = fmaf(b[a], d.h[a], -p);
    float e;
    two_sum(hi, p, hi, e);
    lo += e + pe + b[a] * d.l[a];
  }
  return (hi - rintf(hi)) + lo;
}

}  // namespace
}  // namespace gx
