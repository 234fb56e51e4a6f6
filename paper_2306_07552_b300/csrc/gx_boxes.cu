// The paper's object model (appendix "Additional Collision-Detection
// Details"): resting objects are oriented boxes and a grasped object is
// approximated by a set of spheres.  Here a resting box stands upright
// (centre p, half extents h, yaw about +Y, the robot base's convention:
// x axis (cos, 0, -sin), z axis (sin, 0, cos)); while held it turns with the
// tool (its rotation in the tool frame is fixed at the grasp) and is
// represented for collisions by eight spheres of radius s = min(h) at the
// corners of the box shrunk by s.  Selected per context (gx_config
// object_boxes); the sphere model's kernels are untouched.
//
//   physics_box_kernel: one warp per environment.  Lane i < n_spheres tests
//     robot sphere i against the static grid and every resting box by the
//     exact sphere-box distance in the box's frame; lanes 0..7 test the held
//     box's eight spheres against the grid and the other boxes.  Grasp takes
//     the box nearest the 3 cm tip sphere; release stands the box upright
//     about its current heading, casts its four bottom spheres down (the
//     exact per-cell root of the trilinear field, as for sphere objects) and
//     rests it on the highest landing, unless a cast finds no surface or the
//     box would overlap another (separating axes in the ground plane plus the
//     vertical intervals): then it returns to its pre-grasp pose.
//   reset_box_kernel: one warp per resetting environment; boxes placed in
//     order on support tops by rejection sampling (Philox4x32-10), each try
//     accepted when its eight spheres clear the static grid and it overlaps
//     no box placed before it; then the robot base as in the sphere model.
#include <math_constants.h>

// Compiled twice: as itself (dense grid) and, through gx_boxes_store.cu, with
// GX_STATIC_STORE 1 (box store), whose launchers carry the suffix _store.
#ifndef GX_STATIC_STORE
#define GX_STATIC_STORE 0
#endif
#if GX_STATIC_STORE == 1
#define GX_BOX_LAUNCHER(name) name##_store
#else
#define GX_BOX_LAUNCHER(name) name
#endif

#include "gx_internal.h"
#include "gx_device.cuh"
#include "gx_kin.cuh"

namespace gx {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBoxEnvsPerBlock = 4;
constexpr uint32_t kBoxShapeTag = 0x424F5845u;   // counter word 3 of a box's shape draw
constexpr uint32_t kRobotStreamB = GX_MAX_OBJECTS;
constexpr uint32_t kGoalStreamB = GX_MAX_OBJECTS + 1;

// Exact signed distance from q (box frame) to the box [-h, h].
__device__ __forceinline__ float sd_box(float qx, float qy, float qz, float hx, float hy,
                                        float hz) {
  const float ox = fabsf(qx) - hx, oy = fabsf(qy) - hy, oz = fabsf(qz) - hz;
  const float mx = fmaxf(ox, 0.f), my = fmaxf(oy, 0.f), mz = fmaxf(oz, 0.f);
  return sqrtf(mx * mx + my * my + mz * mz) + fminf(fmaxf(ox, fmaxf(oy, oz)), 0.f);
}

// Distance from c to resting box (o centre, b = (hx, hy, hz, yaw), cs = (cos, sin) of yaw).
__device__ __forceinline__ float box_dist(float4 o, float4 b, float2 cs, float cx, float cy,
                                          float cz) {
  const float dx = cx - o.x, dy = cy - o.y, dz = cz - o.z;
  return sd_box(cs.x * dx - cs.y * dz, dy, cs.y * dx + cs.x * dz, b.x, b.y, b.z);
}

// Two upright boxes overlap iff their vertical intervals overlap and none of
// the four box axes in the ground plane separates their footprints.
__device__ __forceinline__ bool boxes_overlap(float px, float py, float pz, float4 a, float2 ca,
                                              float4 o, float4 b, float2 cb) {
  if (fabsf(py - o.y) >= a.y + b.y) return false;
  const float ax[4][2] = {{ca.x, -ca.y}, {ca.y, ca.x}, {cb.x, -cb.y}, {cb.y, cb.x}};
  const float dx = o.x - px, dz = o.z - pz;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float ux = ax[k][0], uz = ax[k][1];
    const float ra = a.x * fabsf(ux * ax[0][0] + uz * ax[0][1]) + a.z * fabsf(ux * ax[1][0] + uz * ax[1][1]);
    const float rb = b.x * fabsf(ux * ax[2][0] + uz * ax[2][1]) + b.z * fabsf(ux * ax[3][0] + uz * ax[3][1]);
    if (fabsf(dx * ux + dz * uz) >= ra + rb) return false;
  }
  return true;
}

// Carried sphere k of a box with half extents b.xyz: centre in the box frame
// (sign of bit 0 / 1 / 2 of k on x / y / z, clear = minus) and radius.
__device__ __forceinline__ float box_sphere(float4 b, int k, float l[3]) {
  const float s = fminf(b.x, fminf(b.y, b.z));
  l[0] = ((k & 1) ? 1.f : -1.f) * (b.x - s);
  l[1] = ((k & 2) ? 1.f : -1.f) * (b.y - s);
  l[2] = ((k & 4) ? 1.f : -1.f) * (b.z - s);
  return s;
}

// v[lane] from a register array, by selects (no dynamic register indexing).
__device__ __forceinline__ float lane_select(const float v[], int n, int lane) {
  float x = v[0];
#pragma unroll
  for (int k = 1; k < n; ++k) x = lane == k ? v[k] : x;
  return x;
}

__global__ void __launch_bounds__(32 * kBoxEnvsPerBlock) physics_box_kernel(const PhysicsParams P) {
  __shared__ float4 s_obj[kBoxEnvsPerBlock][GX_MAX_OBJECTS];
  __shared__ float4 s_box[kBoxEnvsPerBlock][GX_MAX_OBJECTS];
  __shared__ float2 s_rot[kBoxEnvsPerBlock][GX_MAX_OBJECTS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int env = blockIdx.x * kBoxEnvsPerBlock + w;
  if (blockIdx.x == 0 && threadIdx.x == 0 && P.raster_work) *P.raster_work = 0;
  if (env >= P.n) return;
  const int n = P.n, M = P.M;
  const DScene& S = P.scenes[P.env_scene[env]];
  const gx_robot& rb = P.robot->r;
  float4* so = s_obj[w];
  float4* sb = s_box[w];
  float2* sr = s_rot[w];
  for (int j = lane; j < M; j += 32) {
    so[j] = P.st.obj[(size_t)env * M + j];
    const float4 b = P.st.obox[(size_t)env * M + j];
    sb[j] = b;
    float s, c;
    sincosf(b.w, &s, &c);
    sr[j] = make_float2(c, s);
  }
  __syncwarp();

  // (a1) actions; (a2) candidate pose -- as for sphere objects
  float a = lane < 11 ? P.actions[(size_t)env * 11 + lane] : 0.f;
  const bool bad = lane < 11 && !isfinite(a);
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(P.err, GX_DEV_NONFINITE_ACTION);
  a = bad ? 0.f : clampf(a, -1.f, 1.f);
  float act[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) act[k] = __shfl_sync(kFull, a, k);
  const float x0 = P.st.bx[env], z0 = P.st.bz[env], th0 = P.st.yaw[env];
  float q0[7], cq[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    q0[k] = P.st.q[(size_t)k * n + env];
    cq[k] = clampf(q0[k] + rb.dq_max * act[2 + k], rb.q_min[k], rb.q_max[k]);
  }
  float sth, cth;
  sincosf(th0, &sth, &cth);
  const float cx = x0 + rb.base_step * act[0] * cth;
  const float cz = z0 - rb.base_step * act[0] * sth;
  float cyaw = th0 - rb.base_turn * act[1];
  if (cyaw > CUDART_PI_F) cyaw -= 2.f * CUDART_PI_F;
  if (cyaw <= -CUDART_PI_F) cyaw += 2.f * CUDART_PI_F;
  int held = P.st.held[env];
  if (held >= M) held = -1;
  const int stepc = P.st.step[env] + 1;
  float coff[3] = {P.st.coff[env], P.st.coff[(size_t)n + env], P.st.coff[2 * (size_t)n + env]};
  float roff[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) roff[k] = P.st.roff[(size_t)k * n + env];

  // (a3, a4) FK and sphere centres of the candidate
  const int mylink = lane < rb.n_spheres ? rb.sphere_link[lane] : -1;
  float myR[9], myt[3], eR[9], et[3];
  fk(rb, cx, cz, cyaw, cq, mylink, myR, myt, eR, et);
  __syncwarp();
  const bool active = lane < rb.n_spheres;
  bool cs = false, co = false;
  if (active) {
    float c[3];
    apply(myR, myt, rb.sphere_pos[lane][0], rb.sphere_pos[lane][1], rb.sphere_pos[lane][2], c);
    const float r = rb.sphere_radius[lane];
    float d;
    cs = !grid_query(S, c[0], c[1], c[2], d) || d < r;
    for (int j = 0; j < M; ++j) {
      if (j == held) continue;
      co |= box_dist(so[j], sb[j], sr[j], c[0], c[1], c[2]) < r;
    }
  }
  // the held box's eight spheres at the candidate tool frame
  bool hs = false, ho = false;
  if (held >= 0 && lane < 8) {
    float l[3];
    const float s = box_sphere(sb[held], lane, l);
    float o[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      o[r] = coff[r] + roff[3 * r] * l[0] + roff[3 * r + 1] * l[1] + roff[3 * r + 2] * l[2];
    float c[3];
    apply(eR, et, o[0], o[1], o[2], c);
    float d;
    hs = !grid_query(S, c[0], c[1], c[2], d) || d < s;
    for (int j = 0; j < M; ++j) {
      if (j == held) continue;
      ho |= box_dist(so[j], sb[j], sr[j], c[0], c[1], c[2]) < s;
    }
  }
  const bool hany = __any_sync(kFull, hs || ho);
  const unsigned mask = __ballot_sync(kFull, active && (cs || co)) | (hany ? 1u << 30 : 0u);
  const uint8_t flags = ((__any_sync(kFull, active && cs) || __any_sync(kFull, hs)) ? 1 : 0) |
                        ((__any_sync(kFull, active && co) || __any_sync(kFull, ho)) ? 2 : 0) |
                        (hany ? 4 : 0);

  // (a7) any contact rejects all robot motion
  const bool rev = mask != 0;
  float ax = cx, az = cz, ayaw = cyaw, aq[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) aq[k] = cq[k];
  if (rev) {
    ax = x0; az = z0; ayaw = th0;
#pragma unroll
    for (int k = 0; k < 7; ++k) aq[k] = q0[k];
    fk(rb, ax, az, ayaw, aq, -1, myR, myt, eR, et);
  }

  // (a8) grasp / release at the accepted pose
  int nheld = held;
  uint8_t event = 0;
  float ppre[3] = {P.st.ppre[env], P.st.ppre[(size_t)n + env], P.st.ppre[2 * (size_t)n + env]};
  const bool grasp = act[9] >= 0.5f;
  if (grasp && held < 0) {
    float bs = CUDART_INF_F;
    int bj = -1;
    const float rg = rb.grasp_radius;
    for (int j = lane; j < M; j += 32) {
      const float d = box_dist(so[j], sb[j], sr[j], et[0], et[1], et[2]);
      if (d < rg && d < bs) { bs = d; bj = j; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float os = __shfl_xor_sync(kFull, bs, off);
      const int oj = __shfl_xor_sync(kFull, bj, off);
      if (oj >= 0 && (bj < 0 || os < bs || (os == bs && oj < bj))) { bs = os; bj = oj; }
    }
    if (bj >= 0) {
      // c_off = R_ee^T (p - t_ee), R_off = R_ee^T R_y(yaw)
      const float4 o = so[bj];
      const float2 r2 = sr[bj];
      const float dp[3] = {o.x - et[0], o.y - et[1], o.z - et[2]};
      const float Ry[9] = {r2.x, 0.f, r2.y, 0.f, 1.f, 0.f, -r2.y, 0.f, r2.x};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        coff[r] = eR[r] * dp[0] + eR[3 + r] * dp[1] + eR[6 + r] * dp[2];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          roff[3 * r + c] = eR[r] * Ry[c] + eR[3 + r] * Ry[3 + c] + eR[6 + r] * Ry[6 + c];
      }
      ppre[0] = o.x; ppre[1] = o.y; ppre[2] = o.z;
      nheld = bj;
      event = 1;
    } else {
      event = 2;
    }
  } else if (!grasp && held >= 0) {
    float p[3];
    apply(eR, et, coff[0], coff[1], coff[2], p);
    float R[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        R[3 * r + c] = eR[3 * r] * roff[c] + eR[3 * r + 1] * roff[3 + c] + eR[3 * r + 2] * roff[6 + c];
    // upright about the current heading of the box's x axis (its z axis when
    // x points nearly straight up or down)
    const float yaw = sqrtf(R[0] * R[0] + R[6] * R[6]) >= 1e-3f ? atan2f(-R[6], R[0])
                                                                  : atan2f(R[2], R[8]);
    float sy, cy;
    sincosf(yaw, &sy, &cy);
    const float4 b = sb[held];
    bool ok = true;
    float ytop = -CUDART_INF_F;
    float s = 0.f;
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
      if (k & 2) continue;  // the four bottom spheres
      float l[3];
      s = box_sphere(b, k, l);
      const float bp[3] = {p[0] + cy * l[0] + sy * l[2], p[1] + l[1], p[2] - sy * l[0] + cy * l[2]};
      float y = bp[1];
      ok &= snap_down(S, bp, s + rb.rest_clearance, y, lane);
      ytop = fmaxf(ytop, y);
    }
    const float ly = ytop + (b.y - s);
    const float4 bl = make_float4(b.x, b.y, b.z, yaw);
    const float2 cl = make_float2(cy, sy);
    bool ov = false;
    if (ok)
      for (int m = lane; m < M; m += 32) {
        if (m == held) continue;
        ov |= boxes_overlap(p[0], ly, p[2], bl, cl, so[m], sb[m], sr[m]);
      }
    ov = __any_sync(kFull, ov);
    event = (ok && !ov) ? 3 : 4;
    __syncwarp();
    if (lane == 0) {
      const float rho = so[held].w;
      if (event == 3) {
        so[held] = make_float4(p[0], ly, p[2], rho);
        sb[held] = bl;
        sr[held] = cl;
      } else {
        so[held] = make_float4(ppre[0], ppre[1], ppre[2], rho);
      }
    }
    nheld = -1;
    coff[0] = coff[1] = coff[2] = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) roff[k] = 0.f;
  }
  __syncwarp();
  if (nheld >= 0) {
    float p[3];
    apply(eR, et, coff[0], coff[1], coff[2], p);
    if (lane == 0) so[nheld] = make_float4(p[0], p[1], p[2], so[nheld].w);
    if (P.held_M && lane < 3) {
      // the held box's world rotation times its half extents, for the rasteriser
      const float4 b = sb[nheld];
      float Rr[3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        Rr[c] = eR[3 * lane] * roff[c] + eR[3 * lane + 1] * roff[3 + c] + eR[3 * lane + 2] * roff[6 + c];
      P.held_M[(size_t)env * 3 + lane] = make_float4(Rr[0] * b.x, Rr[1] * b.y, Rr[2] * b.z, 0.f);
    }
  }
  __syncwarp();

  // state write-back
  if (lane == 0) {
    P.st.bx[env] = ax; P.st.bz[env] = az; P.st.yaw[env] = ayaw;
    P.st.held[env] = nheld;
    P.st.step[env] = stepc;
  }
  if (lane < 7) P.st.q[(size_t)lane * n + env] = aq[lane];
  if (lane < 3) {
    P.st.coff[(size_t)lane * n + env] = coff[lane];
    P.st.ppre[(size_t)lane * n + env] = ppre[lane];
  }
  if (lane < 9) P.st.roff[(size_t)lane * n + env] = lane_select(roff, 9, lane);
  for (int j = lane; j < M; j += 32) {
    P.st.obj[(size_t)env * M + j] = so[j];
    P.st.obox[(size_t)env * M + j] = sb[j];
    if (P.out.obj_pos) reinterpret_cast<float4*>(P.out.obj_pos)[(size_t)env * M + j] = so[j];
  }
  // (a9) camera for the rasteriser
  float cam[12];
  camera(rb, ax, az, ayaw, cam);
  if (lane < 12) P.cam[(size_t)env * 12 + lane] = lane_select(cam, 12, lane);
  // (a11) observations other than images
  if (P.out.pose && lane < 16) {
    float v = 0.f;
    if (lane < 7) v = lane_select(aq, 7, lane);
    else if (lane == 7) v = nheld >= 0 ? 1.f : 0.f;
    else if (lane == 8) v = ax;
    else if (lane == 9) v = az;
    else if (lane == 10) v = ayaw;
    else if (lane == 11) v = et[0];
    else if (lane == 12) v = et[1];
    else if (lane == 13) v = et[2];
    else if (lane == 14) v = (float)stepc;
    P.out.pose[(size_t)env * 16 + lane] = v;
  }
  if (lane == 0) {
    if (P.out.held) P.out.held[env] = nheld;
    if (P.out.contact_mask) P.out.contact_mask[env] = mask;
    if (P.out.contact_flags) P.out.contact_flags[env] = flags;
    if (P.out.event) P.out.event[env] = event;
  }
  // rearrangement task: object 0 (a box) is the target, distances between centres
  {
    float* tk = P.st.task + (size_t)env * 16;
    const float tv = lane < 16 ? tk[lane] : 0.f;
    float t16[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) t16[k] = __shfl_sync(kFull, tv, k);
    float C = 0.f;
#pragma unroll
    for (int k = 0; k < 7; ++k) C += (act[2 + k] - t16[6 + k]) * (act[2 + k] - t16[6 + k]);
    float r = -0.001f * C;
    bool success = false;
    float nd = t16[13], ne = t16[14];
    if (M > 0) {
      const float4 o = so[0];
      const float dx = et[0] - o.x, dy = et[1] - o.y, dz = et[2] - o.z;
      const float gx = o.x - t16[0], gy = o.y - t16[1], gz = o.z - t16[2];
      nd = sqrtf(dx * dx + dy * dy + dz * dz);
      ne = sqrtf(gx * gx + gy * gy + gz * gz);
      const bool pick = event == 1 && nheld == 0;
      success = act[10] >= 0.5f && nheld != 0 && ne < 0.15f;
      r += (success ? 10.f : 0.f) + (pick ? 5.f : 0.f) + (t16[13] - nd) + (t16[14] - ne);
    }
    if (lane < 7) tk[6 + lane] = act[2 + lane];
    if (lane == 0) {
      tk[13] = nd;
      tk[14] = ne;
      if (P.out.reward) P.out.reward[env] = r;
      if (P.out.success) P.out.success[env] = success ? 1 : 0;
    }
    if (P.out.task_obs && lane < 12) {
      float syw, cyw;
      sincosf(ayaw, &syw, &cyw);
      const int v = lane / 3, ax3 = lane % 3;
      const float fx = v < 2 ? ax : et[0], fy = v < 2 ? 0.f : et[1], fz = v < 2 ? az : et[2];
      const float tx = (v & 1) ? t16[0] : t16[3], ty = (v & 1) ? t16[1] : t16[4],
                  tz = (v & 1) ? t16[2] : t16[5];
      const float wx = tx - fx, wy = ty - fy, wz = tz - fz;
      P.out.task_obs[(size_t)env * 12 + lane] =
          ax3 == 0 ? cyw * wx - syw * wz : (ax3 == 1 ? wy : syw * wx + cyw * wz);
    }
  }
}

// (a12) masked reset with box objects, one warp per environment (a grid of
// warps strides over the environments).
__global__ void __launch_bounds__(32 * kBoxEnvsPerBlock) reset_box_kernel(const ResetParams P) {
  __shared__ float4 s_obj[kBoxEnvsPerBlock][GX_MAX_OBJECTS];
  __shared__ float4 s_box[kBoxEnvsPerBlock][GX_MAX_OBJECTS];
  __shared__ float2 s_rot[kBoxEnvsPerBlock][GX_MAX_OBJECTS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = P.n, M = P.M;
  const gx_robot& rb = P.robot->r;
  const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
  const float clear = rb.rest_clearance;
  float4* so = s_obj[w];
  float4* sb = s_box[w];
  float2* sr = s_rot[w];
  for (int env = blockIdx.x * kBoxEnvsPerBlock + w; env < n; env += gridDim.x * kBoxEnvsPerBlock) {
    if (P.mask && !P.mask[env]) continue;
    const DScene& S = P.scenes[P.env_scene[env]];
    const uint32_t genv = (uint32_t)(env + P.env_offset);
    const uint32_t ep = (uint32_t)P.st.episode[env] + 1u;
    bool failed = false;
    // 1. boxes in order, tries in order; the lowest accepted try wins, after
    // 64 failures the last try stands
    for (int j = 0; j < M; ++j) {
      const uint4 ws = philox4x32_10(make_uint4(genv, ep, (uint32_t)j, kBoxShapeTag), key);
      const float span = P.rho_max - P.rho_min;
      const float4 hb = make_float4(P.rho_min + unit24(ws.x) * span, P.rho_min + unit24(ws.y) * span,
                                    P.rho_min + unit24(ws.z) * span, 0.f);
      const float rxz = sqrtf(hb.x * hb.x + hb.z * hb.z);
      const float bound = sqrtf(hb.x * hb.x + hb.y * hb.y + hb.z * hb.z);
      float3 p = make_float3(0.f, 0.f, 0.f);
      float yaw = 0.f, cy = 1.f, sy = 0.f;
      bool ok = false;
      for (int t = 0; t < 64 && !ok; ++t) {
        const uint4 wv = philox4x32_10(make_uint4(genv, ep, (uint32_t)j, (uint32_t)t), key);
        const uint32_t si = (uint32_t)(((uint64_t)(wv.x >> 8) * (uint64_t)S.n_supports) >> 24);
        const float* sp = S.supports + 5 * si;
        const float x0 = sp[0] + rxz, x1 = sp[2] - rxz, z0 = sp[1] + rxz, z1 = sp[3] - rxz;
        p = make_float3(x0 + unit24(wv.y) * (x1 - x0), sp[4] + hb.y + clear,
                        z0 + unit24(wv.z) * (z1 - z0));
        yaw = -CUDART_PI_F + unit24(wv.w) * (2.f * CUDART_PI_F);
        sincosf(yaw, &sy, &cy);
        bool badt = false;
        if (lane < 8) {  // lane k: carried sphere k against the static grid
          float l[3];
          const float s = box_sphere(hb, lane, l);
          float d;
          badt = !grid_query(S, p.x + cy * l[0] + sy * l[2], p.y + l[1], p.z - sy * l[0] + cy * l[2], d) ||
                 d < s;
        }
        const float4 bt = make_float4(hb.x, hb.y, hb.z, yaw);
        const float2 ct = make_float2(cy, sy);
        for (int m = lane; m < j; m += 32) badt |= boxes_overlap(p.x, p.y, p.z, bt, ct, so[m], sb[m], sr[m]);
        ok = !__any_sync(kFull, badt);
      }
      failed |= !ok;
      if (lane == 0) {
        so[j] = make_float4(p.x, p.y, p.z, bound);
        sb[j] = make_float4(hb.x, hb.y, hb.z, yaw);
        sr[j] = make_float2(cy, sy);
      }
      __syncwarp();
    }
    // 2. the robot base: every sphere clear of the grid and of every box
    float q[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) q[k] = rb.q_rest[k];
    float bx = 0.f, bz = 0.f, byaw = 0.f;
    bool rok = false;
    for (int t = 0; t < 64 && !rok; ++t) {
      const uint4 wv = philox4x32_10(make_uint4(genv, ep, kRobotStreamB, (uint32_t)t), key);
      robot_try(S, wv, bx, bz, byaw);
      bool hit = false;
      if (lane < rb.n_spheres) {
        float c[3];
        sphere_world(rb, lane, bx, bz, byaw, q, c);
        const float r = rb.sphere_radius[lane];
        float d;
        hit = !grid_query(S, c[0], c[1], c[2], d) || d < r;
        for (int j = 0; j < M && !hit; ++j) hit = box_dist(so[j], sb[j], sr[j], c[0], c[1], c[2]) < r;
      }
      rok = !__any_sync(kFull, hit);
    }
    failed |= !rok;
    if (failed && lane == 0) atomicOr(P.err, GX_DEV_PLACEMENT_FAILED);
    if (lane == 0) {
      P.st.bx[env] = bx; P.st.bz[env] = bz; P.st.yaw[env] = byaw;
      P.st.held[env] = -1;
      P.st.step[env] = 0;
      P.st.episode[env] = (int)ep;
    }
    if (lane < 7) P.st.q[(size_t)lane * n + env] = rb.q_rest[lane];
    if (lane < 3) {
      P.st.coff[(size_t)lane * n + env] = 0.f;
      P.st.ppre[(size_t)lane * n + env] = 0.f;
    }
    if (lane < 9) P.st.roff[(size_t)lane * n + env] = 0.f;
    for (int j = lane; j < M; j += 32) {
      P.st.obj[(size_t)env * M + j] = so[j];
      P.st.obox[(size_t)env * M + j] = sb[j];
    }
    // task: the goal of box 0 on a support top (shrunk by its footprint's
    // circumradius, raised by its half height), first draw of the goal stream
    {
      float task[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) task[k] = 0.f;
      if (M > 0 && S.n_supports > 0) {
        const uint4 wg = philox4x32_10(make_uint4(genv, ep, kGoalStreamB, 0u), key);
        const float4 o = so[0], b = sb[0];
        const float rxz = sqrtf(b.x * b.x + b.z * b.z);
        const uint32_t si = (uint32_t)(((uint64_t)(wg.x >> 8) * (uint64_t)S.n_supports) >> 24);
        const float* sp = S.supports + 5 * si;
        const float x0 = sp[0] + rxz, x1 = sp[2] - rxz, z0 = sp[1] + rxz, z1 = sp[3] - rxz;
        task[0] = x0 + unit24(wg.y) * (x1 - x0);
        task[1] = sp[4] + b.y + clear;
        task[2] = z0 + unit24(wg.z) * (z1 - z0);
        task[3] = o.x;
        task[4] = o.y;
        task[5] = o.z;
        float mR[9], mt[3], eR[9], et[3];
        fk(rb, bx, bz, byaw, q, -1, mR, mt, eR, et);
        const float dx = et[0] - o.x, dy = et[1] - o.y, dz = et[2] - o.z;
        const float gx = o.x - task[0], gy = o.y - task[1], gz = o.z - task[2];
        task[13] = sqrtf(dx * dx + dy * dy + dz * dz);
        task[14] = sqrtf(gx * gx + gy * gy + gz * gz);
      }
      if (lane < 16) P.st.task[(size_t)env * 16 + lane] = lane_select(task, 16, lane);
    }
    float cam[12];
    camera(rb, bx, bz, byaw, cam);
    if (lane < 12) P.cam[(size_t)env * 12 + lane] = lane_select(cam, 12, lane);
    __syncwarp();
  }
}

}  // namespace

void GX_BOX_LAUNCHER(launch_physics_boxes)(const PhysicsParams& p, cudaStream_t s) {
#if GX_STATIC_STORE == 0
  if (p.store) {
    launch_physics_boxes_store(p, s);
    return;
  }
#endif
  const int blocks = (p.n + kBoxEnvsPerBlock - 1) / kBoxEnvsPerBlock;
  physics_box_kernel<<<blocks, 32 * kBoxEnvsPerBlock, 0, s>>>(p);
}

void GX_BOX_LAUNCHER(launch_reset_boxes)(const ResetParams& p, cudaStream_t s) {
#if GX_STATIC_STORE == 0
  if (p.store) {
    launch_reset_boxes_store(p, s);
    return;
  }
#endif
  if (p.n <= 0) return;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int need = (p.n + kBoxEnvsPerBlock - 1) / kBoxEnvsPerBlock;
  const int grid = need < 4 * sms ? need : 4 * sms;
  reset_box_kernel<<<grid, 32 * kBoxEnvsPerBlock, 0, s>>>(p);
}

}  // namespace gx
