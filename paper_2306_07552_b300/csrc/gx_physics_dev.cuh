// Device code of the physics and reset steps of the sphere object model
// (Sec. 3.2), shared by their own kernels (gx_physics.cu) and the fused
// persistent step (gx_fused.cu).  Each including translation unit gets its
// own internal copy.
#pragma once

#include <math_constants.h>

#include <algorithm>

#include "gx_internal.h"
#include "gx_device.cuh"
#include "gx_kin.cuh"

namespace gx {
namespace {
namespace phys {


constexpr unsigned kFull = 0xffffffffu;
constexpr int kEnvsPerBlock = 4;
// Philox streams of a reset beyond the objects' 0..GX_MAX_OBJECTS-1
constexpr uint32_t kRobotStream = GX_MAX_OBJECTS;
constexpr uint32_t kGoalStream = GX_MAX_OBJECTS + 1;

// (a1-a11) one environment's physics step by one warp (lane = sphere);
// so: the warp's shared copy of the environment's objects (GX_MAX_OBJECTS).
__device__ __forceinline__ void physics_env(const PhysicsParams& P, int env, int lane,
                                            float4* so) {
  const int n = P.n, M = P.M;
  const DScene& S = P.scenes[P.env_scene[env]];
  const gx_robot& rb = P.robot->r;
  for (int j = lane; j < M; j += 32) so[j] = P.st.obj[(size_t)env * M + j];

  // (a1) actions, clipped to [-1, 1]; non-finite values count as 0
  float a = lane < 11 ? P.actions[(size_t)env * 11 + lane] : 0.f;
  const bool bad = lane < 11 && !isfinite(a);
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(P.err, GX_DEV_NONFINITE_ACTION);
  a = bad ? 0.f : clampf(a, -1.f, 1.f);
  float act[11];
#pragma unroll
  for (int k = 0; k < 11; ++k) act[k] = __shfl_sync(kFull, a, k);

  // (a2) candidate pose: translate along the pre-step heading, then turn
  // (+1 = clockwise seen from above, so yaw decreases); joints clamped
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
  if (held >= M) held = -1;  // a loaded state cannot index past the objects
  const int stepc = P.st.step[env] + 1;
  float coff[3] = {P.st.coff[env], P.st.coff[(size_t)n + env], P.st.coff[2 * (size_t)n + env]};

  // (a3, a4) FK and sphere centres of the candidate
  const int mylink = lane < rb.n_spheres ? rb.sphere_link[lane] : -1;
  float myR[9], myt[3], eR[9], et[3];
  fk(rb, cx, cz, cyaw, cq, mylink, myR, myt, eR, et);
  __syncwarp();
  bool active = false;
  float c[3] = {0.f, 0.f, 0.f}, r = 0.f;
  if (lane < rb.n_spheres) {
    apply(myR, myt, rb.sphere_pos[lane][0], rb.sphere_pos[lane][1], rb.sphere_pos[lane][2], c);
    r = rb.sphere_radius[lane];
    active = true;
  } else if (lane == 30 && held >= 0) {
    apply(eR, et, coff[0], coff[1], coff[2], c);
    r = so[held].w;
    active = true;
  }
  if (P.nsdf_pass == 1) {  // the neural SDF is queried between the passes
    P.nsdf_pts[(size_t)env * 32 + lane] = make_float4(c[0], c[1], c[2], active ? r : -1.f);
    return;
  }
  // (a5, a6) static grid and free objects (the held object is not tested)
  bool cs = false, co = false, cs_grid = false;
  if (active) {
    float d;
    if (P.nsdf_pass == 2) {
      // learned distance: outside the box is contact; a predicted clearance
      // of at least the margin is free; otherwise (NaN too) the grid decides
      const float dn = P.nsdf_d[(size_t)env * 32 + lane];
      const bool inside = grid_contains(S, c[0], c[1], c[2]);
      const bool trust = inside && dn - r >= P.nsdf_margin;
      cs = !inside || (!trust && (!grid_query(S, c[0], c[1], c[2], d) || d < r));
      if (P.nsdf_counters) {
        cs_grid = !grid_query(S, c[0], c[1], c[2], d) || d < r;
        atomicAdd(P.nsdf_counters + kNsdfSpheres, 1ull);
        if (inside && !trust) atomicAdd(P.nsdf_counters + kNsdfFallbacks, 1ull);
        if (cs != cs_grid) atomicAdd(P.nsdf_counters + kNsdfDisagree, 1ull);
      }
    } else if (P.column) {
      cs = column_contact(S, c[0], c[1], c[2], r);
    } else {
      cs = !grid_query(S, c[0], c[1], c[2], d) || d < r;
    }
    // free objects: with the broad-phase, only those listed in the cell that
    // holds this sphere's XZ disk (held objects stay listed and are skipped)
    const BpCell* cell = P.bp ? bp_cell(P.bp + (size_t)env * 4 * P.bp_cells, P.bp_cells, S, c[0],
                                        c[2], r)
                              : nullptr;
    const int nj = cell ? (int)cell->count : M;
    for (int t = 0; t < nj; ++t) {
      const int j = cell ? (int)cell->id[t] : t;
      if (j == held || j >= M) continue;
      const float4 o = so[j];
      const float dx = c[0] - o.x, dy = c[1] - o.y, dz = c[2] - o.z, rr = r + o.w;
      co |= dx * dx + dy * dy + dz * dz < rr * rr;
    }
  }
  const unsigned mask = __ballot_sync(kFull, active && (cs || co));
  if (P.nsdf_pass == 2 && P.nsdf_counters) {
    const unsigned mask_grid = __ballot_sync(kFull, active && (cs_grid || co));
    if (lane == 0 && mask_grid != mask) atomicAdd(P.nsdf_counters + kNsdfEnvDisagree, 1ull);
  }
  if (P.step_counters) {
    // tests within kNearBand of their threshold (the grid or box store, and
    // the object pairs), counted apart from the decisions above
    bool near_s = false, near_o = false;
    if (active && !P.column) {
      float d;
      if (grid_query(S, c[0], c[1], c[2], d)) near_s = fabsf(d - r) < kNearBand;
      for (int j = 0; j < M; ++j) {
        if (j == held) continue;
        const float4 o = so[j];
        const float dx = c[0] - o.x, dy = c[1] - o.y, dz = c[2] - o.z;
        near_o |= fabsf(sqrtf(dx * dx + dy * dy + dz * dz) - (r + o.w)) < kNearBand;
      }
    }
    const unsigned bs = __ballot_sync(kFull, near_s), bo = __ballot_sync(kFull, near_o);
    if (lane == 0 && bs) atomicAdd(P.step_counters + kStepNearStatic, (unsigned long long)__popc(bs));
    if (lane == 0 && bo) atomicAdd(P.step_counters + kStepNearPairs, (unsigned long long)__popc(bo));
  }
  const unsigned ms = __ballot_sync(kFull, active && cs);
  const unsigned mo = __ballot_sync(kFull, active && co);
  uint8_t flags = (ms ? 1 : 0) | (mo ? 2 : 0) | ((mask >> 30) & 1u ? 4 : 0);

  // (a7) any contact rejects all robot motion this step, unless sliding
  // (appendix "Sliding Heuristic") finds a contact-free base nearby: at most
  // three ground-plane jitters along the penetration-weighted outward
  // normals (horizontal grid gradient; away from object centres), each by
  // the deepest penetration + 1 mm.  Only the base moves, so every sphere
  // translates with it and no new FK is needed.
  bool rev = mask != 0;
  float offx = 0.f, offz = 0.f;
  if (rev && P.slide) {
    bool found = false;
    for (int k = 0; k < 3; ++k) {
      float Dx = 0.f, Dz = 0.f, pen = 0.f;
      const float sx = c[0] + offx, sy = c[1], sz = c[2] + offz;
      if (active) {
        float d, gxx, gzz;
        if (grid_query_grad(S, sx, sy, sz, d, gxx, gzz) && d < r) {
          const float gl = sqrtf(gxx * gxx + gzz * gzz);
          if (gl > 1e-9f) {
            Dx += (r - d) * gxx / gl;
            Dz += (r - d) * gzz / gl;
          }
          pen = fmaxf(pen, r - d);
        }
        for (int j = 0; j < M; ++j) {
          if (j == held) continue;
          const float4 o = so[j];
          const float dx = sx - o.x, dy = sy - o.y, dz = sz - o.z, rr = r + o.w;
          const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
          if (dist < rr) {
            const float vl = sqrtf(dx * dx + dz * dz);
            if (vl > 1e-9f) {
              Dx += (rr - dist) * dx / vl;
              Dz += (rr - dist) * dz / vl;
            }
            pen = fmaxf(pen, rr - dist);
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        Dx += __shfl_xor_sync(kFull, Dx, o);
        Dz += __shfl_xor_sync(kFull, Dz, o);
        pen = fmaxf(pen, __shfl_xor_sync(kFull, pen, o));
      }
      const float dl = sqrtf(Dx * Dx + Dz * Dz);
      if (dl < 1e-5f) break;
      offx += (pen + 0.001f) * Dx / dl;
      offz += (pen + 0.001f) * Dz / dl;
      bool hit = false;
      if (active) {
        const float tx = c[0] + offx, ty = c[1], tz = c[2] + offz;
        float d;
        hit = !grid_query(S, tx, ty, tz, d) || d < r;
        for (int j = 0; j < M && !hit; ++j) {
          if (j == held) continue;
          const float4 o = so[j];
          const float dx = tx - o.x, dy = ty - o.y, dz = tz - o.z, rr = r + o.w;
          hit = dx * dx + dy * dy + dz * dz < rr * rr;
        }
      }
      if (!__any_sync(kFull, hit)) {
        found = true;
        break;
      }
    }
    if (found) {
      rev = false;
      flags |= 8;
    } else {
      offx = offz = 0.f;
    }
  }
  float ax = cx + offx, az = cz + offz, ayaw = cyaw, aq[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) aq[k] = cq[k];
  if (rev) {
    ax = x0; az = z0; ayaw = th0;
#pragma unroll
    for (int k = 0; k < 7; ++k) aq[k] = q0[k];
    fk(rb, ax, az, ayaw, aq, P.robot_sph ? mylink : -1, myR, myt, eR, et);
  } else {
    et[0] += offx;  // a slid base carries the tool frame along
    et[2] += offz;
  }
  if (P.robot_sph) {  // the robot body for the rasteriser: spheres at the accepted pose
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < rb.n_spheres) {
      float cc[3];
      apply(myR, myt, rb.sphere_pos[lane][0], rb.sphere_pos[lane][1], rb.sphere_pos[lane][2], cc);
      v = make_float4(cc[0] + offx, cc[1], cc[2] + offz, rb.sphere_radius[lane]);
    }
    P.robot_sph[(size_t)env * 32 + lane] = v;
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
      const float4 o = so[j];
      const float dx = et[0] - o.x, dy = et[1] - o.y, dz = et[2] - o.z;
      const float d = sqrtf(dx * dx + dy * dy + dz * dz);
      if (d < rg + o.w) {
        const float sd = d - o.w;
        if (sd < bs) { bs = sd; bj = j; }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float os = __shfl_xor_sync(kFull, bs, off);
      const int oj = __shfl_xor_sync(kFull, bj, off);
      if (oj >= 0 && (bj < 0 || os < bs || (os == bs && oj < bj))) { bs = os; bj = oj; }
    }
    if (bj >= 0) {
      const float4 o = so[bj];
      const float dp[3] = {o.x - et[0], o.y - et[1], o.z - et[2]};
#pragma unroll
      for (int k = 0; k < 3; ++k) coff[k] = eR[k] * dp[0] + eR[3 + k] * dp[1] + eR[6 + k] * dp[2];
      ppre[0] = o.x; ppre[1] = o.y; ppre[2] = o.z;
      nheld = bj;
      event = 1;
    } else {
      event = 2;
    }
  } else if (!grasp && held >= 0) {
    float p[3];
    apply(eR, et, coff[0], coff[1], coff[2], p);
    const float rho = so[held].w;
    const float target = rho + rb.rest_clearance;
    float y = p[1];
    const bool ok = snap_down(S, p, target, y, lane);
    bool ov = false;
    if (ok) {
      for (int j = lane; j < M; j += 32) {
        if (j == held) continue;
        const float4 o = so[j];
        const float dx = p[0] - o.x, dy = y - o.y, dz = p[2] - o.z, rr = rho + o.w;
        ov |= dx * dx + dy * dy + dz * dz < rr * rr;
      }
    }
    ov = __any_sync(kFull, ov);
    float lx = p[0], ly = y, lz = p[2];
    event = (ok && !ov) ? 3 : 4;
    if (event == 4 && P.place_jitter) {
      // object placing heuristic (appendix): at most six ground-plane jitters
      // of 2 rho away from the overlapped objects, turned by a uniform angle
      // in [-pi/4, pi/4) (uniform when nothing overlaps), each re-cast down
      // from the release height; Philox on (env, step, k, 0x4A495454)
      const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
      float qx = p[0], qy = y, qz = p[2];
      bool landed = ok;
      for (int k = 0; k < 6; ++k) {
        float Dx = 0.f, Dz = 0.f;
        if (landed) {
          for (int j = lane; j < M; j += 32) {
            if (j == held) continue;
            const float4 o = so[j];
            const float dx = qx - o.x, dy = qy - o.y, dz = qz - o.z;
            if (sqrtf(dx * dx + dy * dy + dz * dz) < rho + o.w) {
              const float vl = sqrtf(dx * dx + dz * dz);
              if (vl > 1e-9f) {
                Dx += dx / vl;
                Dz += dz / vl;
              }
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            Dx += __shfl_xor_sync(kFull, Dx, o);
            Dz += __shfl_xor_sync(kFull, Dz, o);
          }
        }
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)(env + P.env_offset), (uint32_t)(stepc - 1), (uint32_t)k, 0x4A495454u), key);
        const float u = unit24(w.x);
        const float dl = sqrtf(Dx * Dx + Dz * Dz);
        const float phi = dl > 1e-6f ? atan2f(Dz, Dx) + (u - 0.5f) * (0.5f * CUDART_PI_F)
                                     : 2.f * CUDART_PI_F * u;
        float sp, cp;
        sincosf(phi, &sp, &cp);
        qx += 2.f * rho * cp;
        qz += 2.f * rho * sp;
        const float cast[3] = {qx, p[1], qz};
        float y2 = p[1];
        const bool ok2 = snap_down(S, cast, target, y2, lane);
        qy = ok2 ? y2 : p[1];
        landed = ok2;
        bool ov2 = false;
        if (ok2) {
          for (int j = lane; j < M; j += 32) {
            if (j == held) continue;
            const float4 o = so[j];
            const float dx = qx - o.x, dy = qy - o.y, dz = qz - o.z, rr = rho + o.w;
            ov2 |= dx * dx + dy * dy + dz * dz < rr * rr;
          }
        }
        if (ok2 && !__any_sync(kFull, ov2)) {
          lx = qx;
          ly = qy;
          lz = qz;
          event = 5;
          break;
        }
      }
    }
    __syncwarp();
    if (lane == 0) so[held] = event != 4 ? make_float4(lx, ly, lz, rho)
                                         : make_float4(ppre[0], ppre[1], ppre[2], rho);
    if (P.bp && event != 4 && lane == 0) {
      // the object was listed where it rested before the grasp
      BpCell* grids = P.bp + (size_t)env * 4 * P.bp_cells;
      bp_remove(grids, P.bp_cells, S, held, ppre[0], ppre[2], rho);
      bp_insert(grids, P.bp_cells, S, held, lx, lz, rho);
    }
    nheld = -1;
    coff[0] = coff[1] = coff[2] = 0.f;
  }
  __syncwarp();
  if (nheld >= 0 && lane == 0) {
    float p[3];
    apply(eR, et, coff[0], coff[1], coff[2], p);
    so[nheld] = make_float4(p[0], p[1], p[2], so[nheld].w);
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
  for (int j = lane; j < M; j += 32) {
    P.st.obj[(size_t)env * M + j] = so[j];
    if (P.out.obj_pos) reinterpret_cast<float4*>(P.out.obj_pos)[(size_t)env * M + j] = so[j];
  }
  // (a9) camera for the rasteriser
  float cam[12];
  camera(rb, ax, az, ayaw, cam);
  if (lane < 12) {
    float v = cam[0];
#pragma unroll
    for (int k = 1; k < 12; ++k) v = lane == k ? cam[k] : v;
    P.cam[(size_t)env * 12 + lane] = v;
  }
  // (a11) observations other than images
  if (P.out.pose && lane < 16) {
    float v = 0.f;
    if (lane < 7) {
#pragma unroll
      for (int k = 0; k < 7; ++k) v = lane == k ? aq[k] : v;
    } else if (lane == 7) v = nheld >= 0 ? 1.f : 0.f;
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
    if (P.step_counters) {
      unsigned long long* sc = P.step_counters;
      if (mask) atomicAdd(sc + kStepContacts, 1ull);
      if (event == 1) atomicAdd(sc + kStepGrasps, 1ull);
      if (event == 2) atomicAdd(sc + kStepGraspMisses, 1ull);
      if (event == 3 || event == 5) atomicAdd(sc + kStepLanded, 1ull);
      if (event == 4) atomicAdd(sc + kStepRestored, 1ull);
      if (flags & 8) atomicAdd(sc + kStepSlides, 1ull);
    }
  }
  // rearrangement task (App. "Additional Task Details"): object 0 is the
  // target; r = 10 success + 5 pick + (d' - d) + (e' - e) - 0.001 C, d the
  // tip-target and e the target-goal distance (primes: previous step), C the
  // squared change of the 7 joint actions.  Egomotion observations (Sec.
  // 4.1): target start and goal relative to base and tip, base frame.
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
      const int v = lane / 3, a = lane % 3;
      const float fx = v < 2 ? ax : et[0], fy = v < 2 ? 0.f : et[1], fz = v < 2 ? az : et[2];
      const float tx = (v & 1) ? t16[0] : t16[3], ty = (v & 1) ? t16[1] : t16[4],
                  tz = (v & 1) ? t16[2] : t16[5];
      const float wx = tx - fx, wy = ty - fy, wz = tz - fz;
      P.out.task_obs[(size_t)env * 12 + lane] =
          a == 0 ? cyw * wx - syw * wz : (a == 1 ? wy : syw * wx + cyw * wz);
    }
  }
}

// Candidate placement of object j at try t (the same Philox draws the
// sequential definition uses): support by the top 24 bits, uniform on the
// support top shrunk by the radius, resting 1 clearance above it.
__device__ __forceinline__ float3 object_candidate(const DScene& S, uint4 wv, float rho,
                                                   float clear) {
  const uint32_t si = (uint32_t)(((uint64_t)(wv.x >> 8) * (uint64_t)S.n_supports) >> 24);
  const float* sp = S.supports + 5 * si;
  const float x0 = sp[0] + rho, x1 = sp[2] - rho, z0 = sp[1] + rho, z1 = sp[3] - rho;
  return make_float3(x0 + unit24(wv.y) * (x1 - x0), sp[4] + rho + clear, z0 + unit24(wv.z) * (z1 - z0));
}

constexpr int kResetThreads = 256;
constexpr int kTryWindow = 8;  // tries evaluated together before looking further
constexpr int kSerialPlaceMax = 64;  // objects per env placed by the one-warp chain
static_assert(kResetThreads / 32 == kTryWindow, "one warp per try of a window");

// (a12) masked reset, one CTA per environment at a time (the grid strides
// over the environments; CTAs of unmasked ones move on at once): objects on
// support tops, then the robot base in free space, by rejection sampling
// with at most 64 Philox draws each; the lowest accepted try wins, the same
// choice as trying them in order.  Tries are evaluated in windows of 8 so
// that the scene-grid gathers of a window are in flight together (random
// gathers into a multi-gigabyte grid have long latency, and a reset is
// latency-bound):
//   1. the static-scene test of tries 0..7 of every object, all at once;
//   2. objects in order: up to 64 objects by one warp, tries in order (most
//      take their first try, so the chain has no block barrier); more objects
//      in windows of 8 tries, warp w testing try t0 + w; the first try that
//      passed its static test and clears the objects already placed wins;
//   3. every (robot try, sphere) pair of a window at once; the first window
//      with a contact-free try decides.
__device__ void reset_env(const ResetParams& P, int env, float4 (*s_cand)[kTryWindow], float4* so,
                          float* s_rho, unsigned& s_bad, int& s_robot_try) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = P.n, M = P.M;
  const DScene& S = P.scenes[P.env_scene[env]];
  const gx_robot& rb = P.robot->r;
  const uint32_t ep = (uint32_t)P.st.episode[env] + 1u;
  const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
  const float clear = rb.rest_clearance;
  // 1. radii (from each object's try 0) and the first window's static tests
  for (int jt = tid; jt < M * kTryWindow; jt += kResetThreads) {
    const int j = jt / kTryWindow, t = jt % kTryWindow;
    const uint4 w0 = philox4x32_10(make_uint4((uint32_t)(env + P.env_offset), ep, (uint32_t)j, 0u), key);
    const float rho = P.rho_min + unit24(w0.w) * (P.rho_max - P.rho_min);
    if (t == 0) s_rho[j] = rho;
    const uint4 wv = t == 0 ? w0 : philox4x32_10(make_uint4((uint32_t)(env + P.env_offset), ep, (uint32_t)j, (uint32_t)t), key);
    const float3 p = object_candidate(S, wv, rho, clear);
    float d;
    const bool ok = grid_query(S, p.x, p.y, p.z, d) && !(d < rho);
    s_cand[j][t] = make_float4(p.x, p.y, p.z, ok ? 1.f : 0.f);
  }
  if (tid == 0) s_robot_try = -1;
  __syncthreads();
  // 2. objects in order.  Up to kSerialPlaceMax objects (few collisions, most
  // objects take their first try): one warp, tries in order, no block barrier
  // in the chain.  More objects (crowded supports, many tries): windows of 8
  // tries, one per warp, behind block barriers.  Both take the lowest accepted
  // try; after 64 failed tries the last one stands.
  bool failed = false;
  if (M <= kSerialPlaceMax) {
    // warp 0: tries in order (the first 8 from step 1, later ones evaluated by
    // the warp), its lanes splitting each try's test against the placed objects
    if (warp == 0) {
      for (int j = 0; j < M; ++j) {
        const float rho = s_rho[j];
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        bool accepted = false;
        for (int t = 0; t < 64 && !accepted; ++t) {
          if (t < kTryWindow) {
            c = s_cand[j][t];
          } else {
            const uint4 wv =
                philox4x32_10(make_uint4((uint32_t)(env + P.env_offset), ep, (uint32_t)j, (uint32_t)t), key);
            const float3 p = object_candidate(S, wv, rho, clear);
            float d;
            const bool sok = grid_query(S, p.x, p.y, p.z, d) && !(d < rho);
            c = make_float4(p.x, p.y, p.z, sok ? 1.f : 0.f);
          }
          bool hit = false;
          if (c.w > 0.5f)
            for (int k = lane; k < j && !hit; k += 32) {
              const float4 o = so[k];
              const float dx = c.x - o.x, dy = c.y - o.y, dz = c.z - o.z, rr = rho + o.w;
              hit = dx * dx + dy * dy + dz * dz < rr * rr;
            }
          accepted = c.w > 0.5f && !__any_sync(kFull, hit);
        }
        if (lane == 0) so[j] = make_float4(c.x, c.y, c.z, rho);
        __syncwarp();
        failed |= !accepted;
      }
    }
    __syncthreads();
  } else {
    // in each window of tries warp w takes try t0 + w and its lanes split the
    // test against the objects already placed
    for (int j = 0; j < M; ++j) {
      const float rho = s_rho[j];
      int pick_t = -1;
      for (int t0 = 0; t0 < 64 && pick_t < 0; t0 += kTryWindow) {
        const int t = t0 + warp;
        float4 c;
        if (t0 == 0) {
          c = s_cand[j][warp];
        } else {
          const uint4 wv = philox4x32_10(make_uint4((uint32_t)(env + P.env_offset), ep, (uint32_t)j, (uint32_t)t), key);
          const float3 p = object_candidate(S, wv, rho, clear);
          float d;
          const bool sok = grid_query(S, p.x, p.y, p.z, d) && !(d < rho);
          c = make_float4(p.x, p.y, p.z, sok ? 1.f : 0.f);
        }
        bool hit = false;
        if (c.w > 0.5f)
          for (int k = lane; k < j && !hit; k += 32) {
            const float4 o = so[k];
            const float dx = c.x - o.x, dy = c.y - o.y, dz = c.z - o.z, rr = rho + o.w;
            hit = dx * dx + dy * dy + dz * dz < rr * rr;
          }
        const bool ok = c.w > 0.5f && !__any_sync(kFull, hit);
        if (lane == 0) s_cand[j][warp] = c;  // this window's candidates, for the pick below
        if (tid == 0) s_bad = 0u;
        __syncthreads();
        if (lane == 0 && ok) atomicOr(&s_bad, 1u << warp);
        __syncthreads();
        const unsigned okw = s_bad;
        if (okw) pick_t = t0 + __ffs(okw) - 1;
        if (pick_t >= 0 || t0 + kTryWindow >= 64) {
          const int w = pick_t >= 0 ? pick_t - t0 : kTryWindow - 1;
          const float4 cc = s_cand[j][w];
          if (tid == 0) so[j] = make_float4(cc.x, cc.y, cc.z, rho);
        }
        __syncthreads();
      }
      failed |= pick_t < 0;
    }
    __syncthreads();
  }
  if (P.bp) {  // the object broad-phase of this environment, rebuilt
    BpCell* grids = P.bp + (size_t)env * 4 * P.bp_cells;
    uint4* raw = reinterpret_cast<uint4*>(grids);
    for (int i = tid; i < 4 * P.bp_cells; i += kResetThreads) raw[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int j = tid; j < M; j += kResetThreads) bp_insert(grids, P.bp_cells, S, j, so[j].x, so[j].z, so[j].w);
  }
  // 3. robot base, a window of tries at a time
  float q[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) q[k] = rb.q_rest[k];
  const int ns = rb.n_spheres;
  for (int t0 = 0; t0 < 64; t0 += kTryWindow) {
    if (tid == 0) s_bad = 0u;
    __syncthreads();
    for (int p = tid; p < kTryWindow * ns; p += kResetThreads) {
      const int tw = p / ns, i = p - tw * ns;
      const uint4 wv = philox4x32_10(make_uint4((uint32_t)(env + P.env_offset), ep, kRobotStream, (uint32_t)(t0 + tw)), key);
      float x, z, yaw;
      robot_try(S, wv, x, z, yaw);
      float cc[3];
      sphere_world(rb, i, x, z, yaw, q, cc);
      const float r = rb.sphere_radius[i];
      float d;
      bool hit = !grid_query(S, cc[0], cc[1], cc[2], d) || d < r;
      for (int j = 0; j < M && !hit; ++j) {
        const float4 o = so[j];
        const float dx = cc[0] - o.x, dy = cc[1] - o.y, dz = cc[2] - o.z, rr = r + o.w;
        hit = dx * dx + dy * dy + dz * dz < rr * rr;
      }
      if (hit) atomicOr(&s_bad, 1u << tw);
    }
    __syncthreads();
    const unsigned freew = ~s_bad & ((1u << kTryWindow) - 1u);
    // every thread reads this window's word before thread 0 clears it for
    // the next window (without this barrier a late warp could read the
    // cleared word, leave the loop, and miss its share of the next window)
    __syncthreads();
    if (freew) {
      if (tid == 0) s_robot_try = t0 + __ffs(freew) - 1;
      break;
    }
  }
  __syncthreads();
  if (warp != 0) return;
  int t = s_robot_try;
  failed |= t < 0;
  if (t < 0) t = 63;
  const uint4 wv = philox4x32_10(make_uint4((uint32_t)(env + P.env_offset), ep, kRobotStream, (uint32_t)t), key);
  float bx, bz, byaw;
  robot_try(S, wv, bx, bz, byaw);
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
  for (int j = lane; j < M; j += 32) P.st.obj[(size_t)env * M + j] = so[j];
  // task: object 0 is the target; its goal lies on a support top, drawn like
  // an object placement from stream kGoalStream (first draw); previous distances from
  // the episode's first pose, previous joint actions 0
  {
    float task[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) task[k] = 0.f;
    if (M > 0 && S.n_supports > 0) {
      const uint4 wg = philox4x32_10(make_uint4((uint32_t)(env + P.env_offset), ep, kGoalStream, 0u), key);
      const float4 o = so[0];
      const float3 g = object_candidate(S, wg, o.w, rb.rest_clearance);
      task[0] = g.x;
      task[1] = g.y;
      task[2] = g.z;
      task[3] = o.x;
      task[4] = o.y;
      task[5] = o.z;
      float q0[7], mR[9], mt[3], eR[9], et[3];
#pragma unroll
      for (int k = 0; k < 7; ++k) q0[k] = rb.q_rest[k];
      fk(rb, bx, bz, byaw, q0, -1, mR, mt, eR, et);
      const float dx = et[0] - o.x, dy = et[1] - o.y, dz = et[2] - o.z;
      const float gx = o.x - task[0], gy = o.y - task[1], gz = o.z - task[2];
      task[13] = sqrtf(dx * dx + dy * dy + dz * dz);
      task[14] = sqrtf(gx * gx + gy * gy + gz * gz);
    }
    if (lane < 16) {
      float v = task[0];
#pragma unroll
      for (int k = 1; k < 16; ++k) v = lane == k ? task[k] : v;
      P.st.task[(size_t)env * 16 + lane] = v;
    }
  }
  float cam[12];
  camera(rb, bx, bz, byaw, cam);
  if (lane < 12) {
    float v = cam[0];
#pragma unroll
    for (int k = 1; k < 12; ++k) v = lane == k ? cam[k] : v;
    P.cam[(size_t)env * 12 + lane] = v;
  }
}

}  // namespace phys
}  // namespace
}  // namespace gx
