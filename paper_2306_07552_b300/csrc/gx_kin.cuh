// Kinematics shared by the physics and reset kernels of both object models
// (Sec. 3.2): forward kinematics of the arm, the head camera, the
// snap-to-surface cast, and the robot placement tries of a reset.  Included
// by one translation unit per kernel file; each gets its own internal copy.
#pragma once

#include <math_constants.h>

#include "gx_internal.h"
#include "gx_device.cuh"

namespace gx {
namespace {

constexpr unsigned kKinFull = 0xffffffffu;

__device__ __forceinline__ float clampf(float x, float lo, float hi) {
  return fminf(fmaxf(x, lo), hi);
}

// Right-multiplies the row-major rotation R by a rotation of `axis` by the
// angle with sine s, cosine c (columns mix pairwise).  Each case names its
// columns at compile time so R stays in registers.
__device__ __forceinline__ void rmul_axis(float R[9], int axis, float s, float c) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float c0 = R[3 * r], c1 = R[3 * r + 1], c2 = R[3 * r + 2];
    if (axis == 0) {         // Rx: col1' = c col1 + s col2, col2' = -s col1 + c col2
      R[3 * r + 1] = c * c1 + s * c2;
      R[3 * r + 2] = -s * c1 + c * c2;
    } else if (axis == 1) {  // Ry: col0' = c col0 - s col2, col2' = s col0 + c col2
      R[3 * r + 0] = c * c0 - s * c2;
      R[3 * r + 2] = s * c0 + c * c2;
    } else {                 // Rz: col0' = c col0 + s col1, col1' = -s col0 + c col1
      R[3 * r + 0] = c * c0 + s * c1;
      R[3 * r + 1] = -s * c0 + c * c1;
    }
  }
}

__device__ __forceinline__ void apply(const float R[9], const float t[3], float x, float y, float z,
                                      float o[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) o[r] = R[3 * r] * x + R[3 * r + 1] * y + R[3 * r + 2] * z + t[r];
}

// Forward kinematics of the chain (Sec. 3.2).  Returns the frame of link
// `mylink` (0 = base) and the tool-tip frame.
__device__ void fk(const gx_robot& rb, float x, float z, float yaw, const float q[7], int mylink,
                   float myR[9], float myt[3], float eR[9], float et[3]) {
  float s, c;
  sincosf(yaw, &s, &c);
  float R[9] = {c, 0.f, s, 0.f, 1.f, 0.f, -s, 0.f, c};
  float t[3] = {x, 0.f, z};
  if (mylink == 0) {
#pragma unroll
    for (int i = 0; i < 9; ++i) myR[i] = R[i];
    myt[0] = t[0]; myt[1] = t[1]; myt[2] = t[2];
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const float ox = rb.link_offset[k][0], oy = rb.link_offset[k][1], oz = rb.link_offset[k][2];
    float nt[3];
    apply(R, t, ox, oy, oz, nt);
    t[0] = nt[0]; t[1] = nt[1]; t[2] = nt[2];
    float sk, ck;
    sincosf(q[k], &sk, &ck);
    rmul_axis(R, rb.link_axis[k], sk, ck);
    if (mylink == k + 1) {
#pragma unroll
      for (int i = 0; i < 9; ++i) myR[i] = R[i];
      myt[0] = t[0]; myt[1] = t[1]; myt[2] = t[2];
    }
  }
  apply(R, t, rb.link_offset[7][0], rb.link_offset[7][1], rb.link_offset[7][2], et);
#pragma unroll
  for (int i = 0; i < 9; ++i) eR[i] = R[i];
}

// Head camera of base pose (x, z, yaw): R (row-major, columns right, up,
// forward) re-orthonormalised by Gram-Schmidt on forward then up, and eye.
__device__ void camera(const gx_robot& rb, float x, float z, float yaw, float out[12]) {
  float s, c, sp, cp;
  sincosf(yaw, &s, &c);
  sincosf(rb.cam_pitch, &sp, &cp);
  const float R0[9] = {c, 0.f, s, 0.f, 1.f, 0.f, -s, 0.f, c};
  // mount columns in the base frame
  const float Mr[3] = {0.f, 0.f, -1.f}, Mu[3] = {-sp, cp, 0.f}, Mf[3] = {cp, sp, 0.f};
  float r[3], u[3], f[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r[i] = R0[3 * i] * Mr[0] + R0[3 * i + 1] * Mr[1] + R0[3 * i + 2] * Mr[2];
    u[i] = R0[3 * i] * Mu[0] + R0[3 * i + 1] * Mu[1] + R0[3 * i + 2] * Mu[2];
    f[i] = R0[3 * i] * Mf[0] + R0[3 * i + 1] * Mf[1] + R0[3 * i + 2] * Mf[2];
  }
  float nf = rsqrtf(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  f[0] *= nf; f[1] *= nf; f[2] *= nf;
  const float d = u[0] * f[0] + u[1] * f[1] + u[2] * f[2];
  u[0] -= d * f[0]; u[1] -= d * f[1]; u[2] -= d * f[2];
  const float nu = rsqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  u[0] *= nu; u[1] *= nu; u[2] *= nu;
  // right = up x forward
  r[0] = u[1] * f[2] - u[2] * f[1];
  r[1] = u[2] * f[0] - u[0] * f[2];
  r[2] = u[0] * f[1] - u[1] * f[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    out[3 * i + 0] = r[i];
    out[3 * i + 1] = u[i];
    out[3 * i + 2] = f[i];
  }
  float e[3];
  const float t0[3] = {x, 0.f, z};
  apply(R0, t0, rb.cam_pos[0], rb.cam_pos[1], rb.cam_pos[2], e);
  out[9] = e[0]; out[10] = e[1]; out[11] = e[2];
}

// Snap-to-surface: cast a sphere straight down from p; the landing height is
// the highest y <= p.y where the interpolated distance reaches `target`.  At
// fixed (x, z) the field is linear in y between lattice levels, so each
// lane examines one level (32 levels per pass, top down) and the first level
// at or below the target fixes the cell holding the exact root.
__device__ bool snap_down(const DScene& s, const float p[3], float target, float& y, int lane) {
  float d0;
  if (!grid_query(s, p[0], p[1], p[2], d0)) return false;
  if (d0 <= target) {
    y = p[1];
    return true;
  }
  const float gx = (p[0] - s.ox) * s.inv_h, gz = (p[2] - s.oz) * s.inv_h;
  const float gy = (p[1] - s.oy) * s.inv_h;
  const int i = min((int)floorf(gx), s.nx - 2), k = min((int)floorf(gz), s.nz - 2);
  const float tx = gx - i, tz = gz - k;
  const int jstart = min((int)floorf(gy), s.ny - 2);
  float top = p[1], dtop = d0;
  for (int base = jstart; base >= 0; base -= 32) {
    const int j = base - lane;
    float dj = CUDART_INF_F;
    if (j >= 0) {
      const float a0 = gnode(s, i, j, k), a1 = gnode(s, i + 1, j, k);
      const float b0 = gnode(s, i, j, k + 1), b1 = gnode(s, i + 1, j, k + 1);
      const float c0 = a0 + tx * (a1 - a0), c1 = b0 + tx * (b1 - b0);
      dj = c0 + tz * (c1 - c0);
    }
    const unsigned hit = __ballot_sync(kKinFull, j >= 0 && dj <= target);
    if (hit) {
      const int L = __ffs(hit) - 1;
      const float dl = __shfl_sync(kKinFull, dj, L);
      const float dprev = __shfl_sync(kKinFull, dj, L > 0 ? L - 1 : 0);
      const int jr = base - L;
      const float yj = s.oy + (float)jr * s.h;
      const float yt = (L == 0) ? top : s.oy + (float)(jr + 1) * s.h;
      const float dt = (L == 0) ? dtop : dprev;
      y = (yt > yj) ? yj + (target - dl) / (dt - dl) * (yt - yj) : yj;
      return true;
    }
    dtop = __shfl_sync(kKinFull, dj, 31);
    top = s.oy + (float)(base - 31) * s.h;
  }
  return false;
}

__device__ __forceinline__ void robot_try(const DScene& S, uint4 wv, float& x, float& z,
                                          float& yaw) {
  x = S.spawn[0] + unit24(wv.x) * (S.spawn[2] - S.spawn[0]);
  z = S.spawn[1] + unit24(wv.y) * (S.spawn[3] - S.spawn[1]);
  yaw = -CUDART_PI_F + unit24(wv.z) * (2.f * CUDART_PI_F);
}

// World centre of robot sphere i with the base at (x, z, yaw) and joints q:
// the FK chain walked up to the sphere's link.
__device__ void sphere_world(const gx_robot& rb, int i, float x, float z, float yaw,
                             const float q[7], float out[3]) {
  float sn, cs;
  sincosf(yaw, &sn, &cs);
  float R[9] = {cs, 0.f, sn, 0.f, 1.f, 0.f, -sn, 0.f, cs};
  float t[3] = {x, 0.f, z};
  const int link = rb.sphere_link[i];
  for (int k = 0; k < link; ++k) {
    float nt[3];
    apply(R, t, rb.link_offset[k][0], rb.link_offset[k][1], rb.link_offset[k][2], nt);
    t[0] = nt[0]; t[1] = nt[1]; t[2] = nt[2];
    float sk, ck;
    sincosf(q[k], &sk, &ck);
    rmul_axis(R, rb.link_axis[k], sk, ck);
  }
  apply(R, t, rb.sphere_pos[i][0], rb.sphere_pos[i][1], rb.sphere_pos[i][2], out);
}

}  // namespace
}  // namespace gx
