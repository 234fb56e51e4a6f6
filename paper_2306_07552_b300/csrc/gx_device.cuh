// Device functions shared by the step kernels and the neural-SDF kernels:
// the counter-based random generator and the distance-grid query.
#pragma once

#include "gx_internal.h"

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

__device__ __forceinline__ float gnode(const DScene& s, int i, int j, int k) {
  return __ldg(s.grid + ((size_t)k * s.ny + j) * s.nx + i);
}

// Trilinear interpolation at lattice coordinates g (0 <= g <= n - 1 per axis).
__device__ __forceinline__ float grid_lerp(const DScene& s, float gx, float gy, float gz) {
  const int i = min((int)floorf(gx), s.nx - 2);
  const int j = min((int)floorf(gy), s.ny - 2);
  const int k = min((int)floorf(gz), s.nz - 2);
  const float tx = gx - i, ty = gy - j, tz = gz - k;
  const float* g = s.grid + ((size_t)k * s.ny + j) * s.nx + i;
  const size_t sy = s.nx, sz = (size_t)s.nx * s.ny;
  const float c000 = __ldg(g), c100 = __ldg(g + 1);
  const float c010 = __ldg(g + sy), c110 = __ldg(g + sy + 1);
  const float c001 = __ldg(g + sz), c101 = __ldg(g + sz + 1);
  const float c011 = __ldg(g + sz + sy), c111 = __ldg(g + sz + sy + 1);
  const float c00 = c000 + tx * (c100 - c000), c10 = c010 + tx * (c110 - c010);
  const float c01 = c001 + tx * (c101 - c001), c11 = c011 + tx * (c111 - c011);
  const float c0 = c00 + ty * (c10 - c00), c1 = c01 + ty * (c11 - c01);
  return c0 + tz * (c1 - c0);
}

// Trilinear distance and its horizontal gradient (x and z, per metre) at c;
// false outside the lattice box.  d equals grid_query's value.
__device__ bool grid_query_grad(const DScene& s, float cx, float cy, float cz, float& d,
                                float& gxo, float& gzo) {
  const float gx = (cx - s.ox) * s.inv_h, gy = (cy - s.oy) * s.inv_h, gz = (cz - s.oz) * s.inv_h;
  if (!(gx >= 0.f && gx <= (float)(s.nx - 1) && gy >= 0.f && gy <= (float)(s.ny - 1) &&
        gz >= 0.f && gz <= (float)(s.nz - 1)))
    return false;
  d = grid_lerp(s, gx, gy, gz);
  const int i = min((int)floorf(gx), s.nx - 2);
  const int j = min((int)floorf(gy), s.ny - 2);
  const int k = min((int)floorf(gz), s.nz - 2);
  const float tx = gx - i, ty = gy - j, tz = gz - k;
  const float* g = s.grid + ((size_t)k * s.ny + j) * s.nx + i;
  const size_t sy = s.nx, sz = (size_t)s.nx * s.ny;
  const float c000 = __ldg(g), c100 = __ldg(g + 1);
  const float c010 = __ldg(g + sy), c110 = __ldg(g + sy + 1);
  const float c001 = __ldg(g + sz), c101 = __ldg(g + sz + 1);
  const float c011 = __ldg(g + sz + sy), c111 = __ldg(g + sz + sy + 1);
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
