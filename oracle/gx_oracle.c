/*
 * gx_oracle.c -- plain, slow, FP64 reference of the batched environment step
 * of Galactic (arXiv 2306.07552).  TEST INFRASTRUCTURE ONLY (see the header).
 *
 * Every function restates a definition, in the order the method applies it:
 *   action decoding ........ App. A (action space), Sec. 3.2 (offsets applied
 *                            directly to the robot state)
 *   forward kinematics ..... Sec. 3.2 (links placed by FK each step)
 *   static collision ....... Sec. 3.2 / appendix "Collision-Detection
 *                            Details": sphere vs static scene; here the scene
 *                            is a signed-distance grid queried trilinearly
 *   object collision ....... same appendix: robot spheres vs movable objects
 *   resolution ............. Sec. 3.2: a collision disallows all robot
 *                            movement for the step
 *   grasp .................. Sec. 3.2: 3 cm sphere at the end-effector tip
 *   release ................ Sec. 3.2: snap-to-surface by a downward sphere
 *                            cast; appendix "Object Placing Heuristic":
 *                            restore the pre-grasp pose on failure
 *   rendering .............. Sec. 3.1: one egocentric depth + RGB image per
 *                            environment; here the nearest front-facing
 *                            triangle along each pixel-centre ray
 *   reset .................. rejection sampling with Philox4x32-10
 *                            (Salmon et al., SC'11)
 * Nothing here is blocked, fused or reordered beyond those definitions.
 */
#include "gx_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  Ten rounds of the 4x32 S-box with key bumps.  */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in [0, 1) from the top 24 bits: exact in both float and double */
static double unit24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
/* Static scene: signed distance to a union of boxes, sampled on a lattice. */
/* ------------------------------------------------------------------------ */

/* Distance from p to an axis-aligned box: Euclidean distance to the box when
 * outside, minus the distance to the nearest face when inside. */
double orc_box_sdf(const double p[3], const float box[6]) {
  double out2 = 0.0, inmax = -INFINITY;
  for (int a = 0; a < 3; ++a) {
    double lo = box[a], hi = box[a + 3];
    double c = 0.5 * (lo + hi), e = 0.5 * (hi - lo);
    double q = fabs(p[a] - c) - e;
    if (q > 0) out2 += q * q;
    if (q > inmax) inmax = q;
  }
  return sqrt(out2) + (inmax < 0 ? inmax : 0.0);
}

/* Node (i,j,k) of the distance grid: the scene SDF (min over solids) at
 * origin + (i,j,k) * h, computed on demand. */
double orc_grid_node(const orc_scene* s, int i, int j, int k) {
  double p[3] = {(double)s->grid_origin[0] + i * (double)s->grid_h,
                 (double)s->grid_origin[1] + j * (double)s->grid_h,
                 (double)s->grid_origin[2] + k * (double)s->grid_h};
  double d = INFINITY;
  for (int b = 0; b < s->n_boxes; ++b) {
    double v = orc_box_sdf(p, s->boxes + 6 * b);
    if (v < d) d = v;
  }
  return d;
}

/* Trilinear interpolation of the node values at c.  Returns 0 when c lies
 * outside the lattice box (that counts as contact); *edge receives the
 * distance from c to the lattice boundary (negative outside). */
int orc_grid_query(const orc_scene* s, const double c[3], double* d, double* edge) {
  double h = s->grid_h, g[3], t[3];
  int i[3];
  double e = INFINITY;
  for (int a = 0; a < 3; ++a) {
    g[a] = (c[a] - (double)s->grid_origin[a]) / h;
    double ea = fmin(g[a], (double)(s->grid_dims[a] - 1) - g[a]) * h;
    if (ea < e) e = ea;
  }
  if (edge) *edge = e;
  if (e < 0) return 0;
  for (int a = 0; a < 3; ++a) {
    i[a] = (int)floor(g[a]);
    if (i[a] > s->grid_dims[a] - 2) i[a] = s->grid_dims[a] - 2;
    t[a] = g[a] - i[a];
  }
  double v = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? t[0] : 1 - t[0]) * (dy ? t[1] : 1 - t[1]) * (dz ? t[2] : 1 - t[2]);
        v += w * orc_grid_node(s, i[0] + dx, i[1] + dy, i[2] + dz);
      }
  *d = v;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Column grid (appendix "Additional Collision-Detection Details"): for each */
/* radius R of the working set {1.5, 5, 12} cm, a lattice of vertical       */
/* columns 3 cm apart in XZ over the grid box (column (i, k) at origin +    */
/* (i, k) * 3 cm); each column holds the free spans of the centre height y  */
/* of a sphere of radius R: [oy, oy + (ny-1) h] minus, for every box whose  */
/* XZ rectangle lies closer than R to the column, the open interval         */
/* (y0 - e, y1 + e) with e = sqrt(R^2 - dxz^2).  A sphere of radius r is    */
/* tested with the smallest R >= r (1e-5 relative tolerance) at the nearest */
/* column: contact unless its centre height lies in a free span widened by  */
/* R - r at both ends; a centre outside the columns' extent is contact.     */
/* ------------------------------------------------------------------------ */
static const double ORC_COL_R[3] = {0.015, 0.05, 0.12};
#define ORC_COL_S 0.03
#define ORC_COL_CAP 64

int orc_column_radius_index(double r) {
  for (int k = 0; k < 3; ++k)
    if (r <= ORC_COL_R[k] * (1.0 + 1e-5)) return k;
  return 2;
}

void orc_column_dims(const orc_scene* s, int32_t dims[2]) {
  dims[0] = (int)floor((s->grid_dims[0] - 1) * (double)s->grid_h / ORC_COL_S + 1e-6) + 1;
  dims[1] = (int)floor((s->grid_dims[2] - 1) * (double)s->grid_h / ORC_COL_S + 1e-6) + 1;
}

int orc_column_spans(const orc_scene* s, int ri, int i, int k, double spans[][2], int cap) {
  const double R = ORC_COL_R[ri];
  const double x = (double)s->grid_origin[0] + i * ORC_COL_S;
  const double z = (double)s->grid_origin[2] + k * ORC_COL_S;
  const double ylo = (double)s->grid_origin[1];
  const double yhi = ylo + (s->grid_dims[1] - 1) * (double)s->grid_h;
  double iv[ORC_COL_CAP][2];
  int n = 0;
  for (int b = 0; b < s->n_boxes && n < ORC_COL_CAP; ++b) {
    const float* bx = s->boxes + 6 * b;
    double dx = fmax(fmax((double)bx[0] - x, 0.0), x - (double)bx[3]);
    double dz = fmax(fmax((double)bx[2] - z, 0.0), z - (double)bx[5]);
    double d2 = dx * dx + dz * dz;
    if (d2 >= R * R) continue;
    double e = sqrt(R * R - d2);
    double lo = (double)bx[1] - e, hi = (double)bx[4] + e;
    if (hi <= ylo || lo >= yhi) continue;
    /* insertion by lower end */
    int m = n++;
    while (m > 0 && iv[m - 1][0] > lo) {
      iv[m][0] = iv[m - 1][0];
      iv[m][1] = iv[m - 1][1];
      --m;
    }
    iv[m][0] = lo;
    iv[m][1] = hi;
  }
  int ns = 0;
  double cur = ylo;
  for (int t = 0; t < n; ++t) {
    if (iv[t][0] > cur && ns < cap) {
      spans[ns][0] = cur;
      spans[ns][1] = iv[t][0];
      ns++;
    }
    if (iv[t][1] > cur) cur = iv[t][1];
  }
  if (cur <= yhi && ns < cap) {
    spans[ns][0] = cur;
    spans[ns][1] = yhi;
    ns++;
  }
  return ns;
}

int orc_column_contact(const orc_scene* s, const double c[3], double r, int* nb) {
  int32_t dims[2];
  orc_column_dims(s, dims);
  const double fi = (c[0] - (double)s->grid_origin[0]) / ORC_COL_S;
  const double fk = (c[2] - (double)s->grid_origin[2]) / ORC_COL_S;
  /* nearest-column choice: near band within 1e-5 m of a column boundary
   * (FP32 and FP64 sphere centres agree to a few 1e-6 m) */
  if (fabs(fi - floor(fi) - 0.5) < 1e-5 / ORC_COL_S) (*nb)++;
  if (fabs(fk - floor(fk) - 0.5) < 1e-5 / ORC_COL_S) (*nb)++;
  const int i = (int)floor(fi + 0.5), k = (int)floor(fk + 0.5);
  if (i < 0 || i >= dims[0] || k < 0 || k >= dims[1]) return 1;
  double sp[ORC_COL_CAP][2];
  const int ri = orc_column_radius_index(r);
  const int n = orc_column_spans(s, ri, i, k, sp, ORC_COL_CAP);
  /* the spans are for radius R >= r: widened by R - r at both ends (exact
   * for surfaces directly above or below the column, conservative beside
   * walls, which block the whole column within R) */
  const double w = ORC_COL_R[ri] > r ? ORC_COL_R[ri] - r : 0.0;
  int free_ = 0;
  for (int t = 0; t < n; ++t) {
    const double lo = sp[t][0] - w, hi = sp[t][1] + w;
    if (fabs(c[1] - lo) < ORC_BAND || fabs(c[1] - hi) < ORC_BAND) (*nb)++;
    if (c[1] >= lo && c[1] <= hi) free_ = 1;
  }
  return !free_;
}

/* Gradient of the trilinear interpolant at c (the cell the query above
 * uses), per metre; 0 outside the lattice box. */
int orc_grid_gradient(const orc_scene* s, const double c[3], double g[3]) {
  double h = s->grid_h, gl[3], t[3];
  int i[3];
  g[0] = g[1] = g[2] = 0.0;
  for (int a = 0; a < 3; ++a) {
    gl[a] = (c[a] - (double)s->grid_origin[a]) / h;
    if (gl[a] < 0 || gl[a] > s->grid_dims[a] - 1) return 0;
    i[a] = (int)floor(gl[a]);
    if (i[a] > s->grid_dims[a] - 2) i[a] = s->grid_dims[a] - 2;
    t[a] = gl[a] - i[a];
  }
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double v = orc_grid_node(s, i[0] + dx, i[1] + dy, i[2] + dz);
        double wx = dx ? t[0] : 1 - t[0], wy = dy ? t[1] : 1 - t[1], wz = dz ? t[2] : 1 - t[2];
        double sx = dx ? 1.0 : -1.0, sy = dy ? 1.0 : -1.0, sz = dz ? 1.0 : -1.0;
        g[0] += sx * wy * wz * v / h;
        g[1] += wx * sy * wz * v / h;
        g[2] += wx * wy * sz * v / h;
      }
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Rigid frames: R row-major 3x3 then t; x_world = R x_local + t.           */
/* ------------------------------------------------------------------------ */
static void fr_ident(double F[12]) {
  memset(F, 0, 12 * sizeof(double));
  F[0] = F[4] = F[8] = 1.0;
}
static void fr_mul(const double A[12], const double B[12], double O[12]) {
  double T[12];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      T[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
    T[9 + r] = A[3 * r] * B[9] + A[3 * r + 1] * B[10] + A[3 * r + 2] * B[11] + A[9 + r];
  }
  memcpy(O, T, sizeof(T));
}
static void fr_trans(double F[12], double x, double y, double z) {
  fr_ident(F);
  F[9] = x; F[10] = y; F[11] = z;
}
static void fr_rot(double F[12], int axis, double a) {
  double c = cos(a), s = sin(a);
  fr_ident(F);
  if (axis == 0) { F[4] = c; F[5] = -s; F[7] = s; F[8] = c; }
  else if (axis == 1) { F[0] = c; F[2] = s; F[6] = -s; F[8] = c; }
  else { F[0] = c; F[1] = -s; F[3] = s; F[4] = c; }
}
static void fr_apply(const double F[12], const double p[3], double o[3]) {
  for (int r = 0; r < 3; ++r) o[r] = F[3 * r] * p[0] + F[3 * r + 1] * p[1] + F[3 * r + 2] * p[2] + F[9 + r];
}

/* Forward kinematics (Sec. 3.2).  Base frame T0 = Trans(x,0,z) Ry(yaw);
 * T_k = T_{k-1} Trans(o_k) Rot(axis_k, q_k); tool tip = T_7 Trans(o_tip);
 * head camera = T0 Trans(cam_pos) M where M has columns right = (0,0,-1),
 * up = (-sin p, cos p, 0), forward = (cos p, sin p, 0) for pitch p. */
void orc_fk(const orc_robot* rb, const double base[3], const double q[7], double links[8][12],
            double ee[12], double cam[12]) {
  double A[12], B[12];
  fr_trans(A, base[0], 0.0, base[1]);
  fr_rot(B, 1, base[2]);
  fr_mul(A, B, links[0]);
  for (int k = 1; k <= 7; ++k) {
    const float* o = rb->link_offset + 3 * (k - 1);
    fr_trans(A, o[0], o[1], o[2]);
    fr_mul(links[k - 1], A, B);
    fr_rot(A, rb->link_axis[k - 1], q[k - 1]);
    fr_mul(B, A, links[k]);
  }
  if (ee) {
    const float* o = rb->link_offset + 21;
    fr_trans(A, o[0], o[1], o[2]);
    fr_mul(links[7], A, ee);
  }
  if (cam) {
    double p = rb->cam_pitch, M[12];
    double sp = sin(p), cp = cos(p);
    /* columns: right, up, forward */
    M[0] = 0.0; M[1] = -sp; M[2] = cp;
    M[3] = 0.0; M[4] = cp;  M[5] = sp;
    M[6] = -1.0; M[7] = 0.0; M[8] = 0.0;
    M[9] = rb->cam_pos[0]; M[10] = rb->cam_pos[1]; M[11] = rb->cam_pos[2];
    fr_mul(links[0], M, cam);
  }
}

void orc_sphere_centres(const orc_robot* rb, const double base[3], const double q[7],
                        double out[][3]) {
  double links[8][12];
  orc_fk(rb, base, q, links, NULL, NULL);
  for (int i = 0; i < rb->n_spheres; ++i) {
    double p[3] = {rb->sphere_pos[3 * i], rb->sphere_pos[3 * i + 1], rb->sphere_pos[3 * i + 2]};
    fr_apply(links[rb->sphere_link[i]], p, out[i]);
  }
}

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static double dist3(const double a[3], const double b[3]) {
  double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Yaw kept in (-pi, pi]. */
static double wrap_pi(double a) {
  while (a > PI) a -= 2 * PI;
  while (a <= -PI) a += 2 * PI;
  return a;
}

/* Static contact of a sphere (c, r): outside the lattice, or d(c) < r. */
static int static_contact(const orc_scene* s, const double c[3], double r, int* nb) {
  double d, edge;
  int inside = orc_grid_query(s, c, &d, &edge);
  if (fabs(edge) < ORC_BAND) (*nb)++;
  if (!inside) return 1;
  if (fabs(d - r) < ORC_BAND) (*nb)++;
  return d < r;
}

static int pair_contact(const double a[3], double ra, const double b[3], double rb_, int* nb) {
  double d = dist3(a, b);
  if (fabs(d - (ra + rb_)) < ORC_BAND) (*nb)++;
  return d < ra + rb_;
}

/* Snap-to-surface (Sec. 3.2): cast the sphere straight down from p and
 * return the highest y <= p.y where the interpolated distance reaches
 * `target` (= radius + resting clearance).  At fixed (x, z) the trilinear
 * field is linear in y inside each cell, so the landing height is the exact
 * root of that line in the first cell (walking down) whose lower value is at
 * or below the target.  *ok = 0 when no such height exists in the lattice. */
double orc_snap(const orc_scene* s, const double p[3], double target, int* ok, int* nb) {
  double h = s->grid_h;
  double d0, edge;
  *ok = 0;
  if (!orc_grid_query(s, p, &d0, &edge)) {
    if (fabs(edge) < ORC_BAND) (*nb)++;
    return p[1];
  }
  if (fabs(edge) < ORC_BAND) (*nb)++;
  if (fabs(d0 - target) < ORC_BAND) (*nb)++;
  if (d0 <= target) { *ok = 1; return p[1]; }
  /* level j lies at y_j = origin_y + j h; the start cell is the one the
   * trilinear query above used for p. */
  double gy = (p[1] - (double)s->grid_origin[1]) / h;
  int j = (int)floor(gy);
  if (j > s->grid_dims[1] - 2) j = s->grid_dims[1] - 2;
  double top = p[1], dtop = d0;
  for (; j >= 0; --j) {
    double yj = (double)s->grid_origin[1] + j * h;
    double q[3] = {p[0], yj, p[2]};
    double dj, e2;
    orc_grid_query(s, q, &dj, &e2);
    if (fabs(dj - target) < ORC_BAND) (*nb)++;
    if (dj <= target) {
      /* linear root between (yj, dj) and (top, dtop) */
      double slope = (dtop - dj) / (top - yj > 0 ? top - yj : 1.0);
      if (slope < 0.05) (*nb)++; /* flat crossing: height sensitive to rounding */
      double y = (top > yj) ? yj + (target - dj) / (dtop - dj) * (top - yj) : yj;
      *ok = 1;
      return y;
    }
    top = yj;
    dtop = dj;
  }
  return p[1];
}

/* ------------------------------------------------------------------------ */
/* One environment step (Sec. 3.2, App. A).                                 */
/* ------------------------------------------------------------------------ */
/* Static test with a learned distance (the workload's neural SDF): a centre
 * outside the lattice box is in contact; a predicted clearance dhat - r of at
 * least `margin` is free without consulting the grid; otherwise the grid
 * decides.  Predictions within `band` of the margin count as near band. */
static int neural_static_contact(const orc_scene* s, const double c[3], double r, double dhat,
                                 double margin, double band, int* nb) {
  double d, edge;
  int inside = orc_grid_query(s, c, &d, &edge);
  if (fabs(edge) < ORC_BAND) (*nb)++;
  if (!inside) return 1;
  if (fabs(dhat - r - margin) < band) (*nb)++;
  if (dhat - r >= margin) return 0;
  if (fabs(d - r) < ORC_BAND) (*nb)++;
  return d < r;
}

static void candidate_pose(const orc_robot* rb, const orc_state* st, const double a[11],
                           double cb[3], double cq[7]) {
  /* translate along the pre-step heading, then turn; +1 on the turn action
   * is clockwise seen from above (yaw decreases). */
  double th = st->base[2];
  cb[0] = st->base[0] + (double)rb->base_step * a[0] * cos(th);
  cb[1] = st->base[1] - (double)rb->base_step * a[0] * sin(th);
  cb[2] = wrap_pi(th - (double)rb->base_turn * a[1]);
  for (int k = 0; k < 7; ++k)
    cq[k] = clampd(st->q[k] + (double)rb->dq_max * a[2 + k], rb->q_min[k], rb->q_max[k]);
}

static void clip_actions(const float act[11], double a[11]) {
  for (int k = 0; k < 11; ++k) a[k] = isfinite(act[k]) ? clampd(act[k], -1.0, 1.0) : 0.0;
}

void orc_candidate_spheres(const orc_robot* rb, const orc_state* st, const float act[11],
                           double c[31][3], double r[31], int32_t active[31]) {
  double a[11], cb[3], cq[7], links[8][12], ee[12];
  clip_actions(act, a);
  candidate_pose(rb, st, a, cb, cq);
  orc_fk(rb, cb, cq, links, ee, NULL);
  for (int i = 0; i < 31; ++i) { active[i] = 0; r[i] = 0; c[i][0] = c[i][1] = c[i][2] = 0; }
  for (int i = 0; i < rb->n_spheres; ++i) {
    double p[3] = {rb->sphere_pos[3 * i], rb->sphere_pos[3 * i + 1], rb->sphere_pos[3 * i + 2]};
    fr_apply(links[rb->sphere_link[i]], p, c[i]);
    r[i] = rb->sphere_radius[i];
    active[i] = 1;
  }
  if (st->held >= 0) {
    fr_apply(ee, st->c_off, c[30]);
    r[30] = st->obj[st->held][3];
    active[30] = 1;
  }
}

void orc_step(const orc_robot* rb, const orc_scene* sc, orc_state* st, const float act[11],
              orc_step_out* out) {
  orc_step_opts o;
  memset(&o, 0, sizeof(o));
  orc_step_ex(rb, sc, st, act, &o, out);
}

void orc_step_nsdf(const orc_robot* rb, const orc_scene* sc, orc_state* st, const float act[11],
                   const double* dhat, double margin, double band, orc_step_out* out) {
  orc_step_opts o;
  memset(&o, 0, sizeof(o));
  o.dhat = dhat;
  o.margin = margin;
  o.band = band;
  orc_step_ex(rb, sc, st, act, &o, out);
}

/* Contacts of the robot spheres cs[0..n) and the held object ph (when h >=
 * 0) shifted by (ox, 0, oz), grid rule, counting near-band decisions. */
static uint32_t shifted_contacts(const orc_robot* rb, const orc_scene* sc, const orc_state* st,
                                 double cs[][3], const double ph[3], double ox, double oz, int* nb) {
  uint32_t m = 0;
  int h = st->held;
  for (int i = 0; i <= 30; ++i) {
    if (i >= rb->n_spheres && !(i == 30 && h >= 0)) continue;
    const double* c0 = i == 30 ? ph : cs[i];
    double c[3] = {c0[0] + ox, c0[1], c0[2] + oz};
    double r = i == 30 ? st->obj[h][3] : rb->sphere_radius[i];
    int hit = static_contact(sc, c, r, nb);
    for (int j = 0; j < st->n_obj && !hit; ++j)
      if (j != h && pair_contact(c, r, st->obj[j], st->obj[j][3], nb)) hit = 1;
    if (hit) m |= 1u << i;
  }
  return m;
}

/* Sliding heuristic (appendix "Sliding Heuristic"): from the candidate pose,
 * at most three jitters of the base in the ground plane.  Direction: the sum
 * over penetrating spheres of penetration x outward ground-plane normal (the
 * horizontal gradient of the distance field for the static scene, away from
 * the object's centre for objects), normalised; length: the deepest
 * penetration + 1 mm.  A zero direction (|sum| < 1e-5 m) ends the search.
 * Returns 1 and the base shift when a contact-free pose was found. */
static int slide_search(const orc_robot* rb, const orc_scene* sc, const orc_state* st,
                        double cs[][3], const double ph[3], double off[2], int* nb) {
  int h = st->held;
  off[0] = off[1] = 0.0;
  for (int k = 0; k < 3; ++k) {
    double D[2] = {0.0, 0.0}, pen = 0.0;
    for (int i = 0; i <= 30; ++i) {
      if (i >= rb->n_spheres && !(i == 30 && h >= 0)) continue;
      const double* c0 = i == 30 ? ph : cs[i];
      double c[3] = {c0[0] + off[0], c0[1], c0[2] + off[1]};
      double r = i == 30 ? st->obj[h][3] : rb->sphere_radius[i];
      double d, edge, g[3];
      if (orc_grid_query(sc, c, &d, &edge) && d < r) {
        orc_grid_gradient(sc, c, g);
        double gl = sqrt(g[0] * g[0] + g[2] * g[2]);
        if (gl > 1e-9) {
          D[0] += (r - d) * g[0] / gl;
          D[1] += (r - d) * g[2] / gl;
        }
        if (r - d > pen) pen = r - d;
      }
      for (int j = 0; j < st->n_obj; ++j) {
        if (j == h) continue;
        double dist = dist3(c, st->obj[j]), rr = r + st->obj[j][3];
        if (dist < rr) {
          double vx = c[0] - st->obj[j][0], vz = c[2] - st->obj[j][2], vl = sqrt(vx * vx + vz * vz);
          if (vl > 1e-9) {
            D[0] += (rr - dist) * vx / vl;
            D[1] += (rr - dist) * vz / vl;
          }
          if (rr - dist > pen) pen = rr - dist;
        }
      }
    }
    double dl = sqrt(D[0] * D[0] + D[1] * D[1]);
    if (dl < 1e-4) (*nb)++;
    if (dl < 1e-5) return 0;
    off[0] += (pen + 0.001) * D[0] / dl;
    off[1] += (pen + 0.001) * D[1] / dl;
    if (shifted_contacts(rb, sc, st, cs, ph, off[0], off[1], nb) == 0) return 1;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Oriented boxes (appendix "Additional Collision-Detection Details": the   */
/* paper's resting objects are oriented boxes and a grasped object is a set */
/* of spheres).  A resting box stands upright: centre p, half extents h,    */
/* rotation R_y(yaw) (the robot base's convention: x axis (cos, 0, -sin),   */
/* z axis (sin, 0, cos)).                                                   */
/* ------------------------------------------------------------------------ */
void orc_box_local(const double p[3], double yaw, const double c[3], double q[3]) {
  /* q = R_y(yaw)^T (c - p) */
  const double cy = cos(yaw), sy = sin(yaw);
  const double dx = c[0] - p[0], dy = c[1] - p[1], dz = c[2] - p[2];
  q[0] = cy * dx - sy * dz;
  q[1] = dy;
  q[2] = sy * dx + cy * dz;
}

/* Exact signed distance from q (box frame) to the box [-h, h]. */
static double sd_box_local(const double q[3], const double h[3]) {
  double o[3], out = 0.0, in = -INFINITY;
  for (int a = 0; a < 3; ++a) {
    o[a] = fabs(q[a]) - h[a];
    if (o[a] > 0) out += o[a] * o[a];
    if (o[a] > in) in = o[a];
  }
  return sqrt(out) + (in < 0 ? in : 0.0);
}

double orc_box_distance(const orc_state* st, int j, const double c[3]) {
  double q[3];
  orc_box_local(st->obj[j], st->box[j][3], c, q);
  return sd_box_local(q, st->box[j]);
}

static int sphere_box_contact(const orc_state* st, int j, const double c[3], double r, int* nb) {
  const double d = orc_box_distance(st, j, c);
  if (fabs(d - r) < ORC_BAND) (*nb)++;
  return d < r;
}

/* The eight carried spheres: radius s = min(h), centres at the corners of
 * the box shrunk by s, (+-(hx-s), +-(hy-s), +-(hz-s)); corner k has the
 * signs of bits 0 (x), 1 (y), 2 (z) of k (bit clear = minus). */
double orc_box_spheres(const double h[3], double centres[8][3]) {
  const double s = fmin(h[0], fmin(h[1], h[2]));
  for (int k = 0; k < 8; ++k)
    for (int a = 0; a < 3; ++a) centres[k][a] = ((k >> a) & 1 ? 1.0 : -1.0) * (h[a] - s);
  return s;
}

/* Two upright boxes overlap iff their vertical intervals overlap and no
 * ground-plane axis among the four box axes separates their footprints
 * (separating-axis theorem for convex polygons); touching is not overlap. */
int orc_boxes_overlap(const double pa[3], const double ba[4], const double pb[3],
                      const double bb[4], int* nb) {
  const double gy = fabs(pa[1] - pb[1]) - (ba[1] + bb[1]);
  if (fabs(gy) < ORC_BAND) (*nb)++;
  if (gy >= 0) return 0;
  const double ax[4][2] = {{cos(ba[3]), -sin(ba[3])}, {sin(ba[3]), cos(ba[3])},
                           {cos(bb[3]), -sin(bb[3])}, {sin(bb[3]), cos(bb[3])}};
  const double d[2] = {pb[0] - pa[0], pb[2] - pa[2]};
  double sep = -INFINITY;
  for (int k = 0; k < 4; ++k) {
    const double* u = ax[k];
    const double ra = ba[0] * fabs(u[0] * ax[0][0] + u[1] * ax[0][1]) +
                      ba[2] * fabs(u[0] * ax[1][0] + u[1] * ax[1][1]);
    const double rb_ = bb[0] * fabs(u[0] * ax[2][0] + u[1] * ax[2][1]) +
                       bb[2] * fabs(u[0] * ax[3][0] + u[1] * ax[3][1]);
    const double sk = fabs(d[0] * u[0] + d[1] * u[1]) - (ra + rb_);
    if (sk > sep) sep = sk;
  }
  if (fabs(sep) < ORC_BAND) (*nb)++;
  return sep < 0;
}

/* World rotation of object j: R_y(yaw) resting, R_ee R_off while held. */
static void box_rotation(const orc_state* st, int j, const double ee[12], double R[9]) {
  if (j == st->held) {
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        R[3 * r + c] = ee[3 * r] * st->r_off[c] + ee[3 * r + 1] * st->r_off[3 + c] +
                       ee[3 * r + 2] * st->r_off[6 + c];
  } else {
    const double cy = cos(st->box[j][3]), sy = sin(st->box[j][3]);
    const double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
    memcpy(R, Ry, sizeof(Ry));
  }
}

/* Upright yaw of a box with world rotation R: the heading of its x axis in
 * the ground plane, or of its z axis when the x axis points (nearly) up. */
static double upright_yaw(const double R[9], int* nb) {
  const double hx = hypot(R[0], R[6]);
  if (fabs(hx - 1e-3) < ORC_BAND) (*nb)++;
  if (hx >= 1e-3) return atan2(-R[6], R[0]);
  return atan2(R[2], R[8]);
}

/* Reward of the rearrangement task and the egomotion observations, after
 * the step's motion and grasp/release (st updated, ee the tool frame at the
 * accepted pose, event the step's grasp event). */
static void task_epilogue(orc_state* st, const double a[11], const double ee[12], uint8_t event,
                          orc_step_out* out, int* nbp) {
  int nb = 0;
  /* reward of the rearrangement task (App. "Additional Task Details"):
   *   r = 10 I_success + 5 I_pick + (d_{t-1} - d_t) + (e_{t-1} - e_t) - 0.001 C_t
   * with d the tip-target distance, e the target-goal distance, C_t the
   * squared change of the 7 joint actions; success = stop called while the
   * target rests within 15 cm of the goal; pick = the target just grasped.
   * Egomotion observations (Sec. 4.1): the target's start and the goal
   * relative to the base and to the tool tip, in the base frame. */
  {
    const double tip[3] = {ee[9], ee[10], ee[11]};
    double C = 0.0;
    for (int k = 0; k < 7; ++k) C += (a[2 + k] - st->prev_a[k]) * (a[2 + k] - st->prev_a[k]);
    double r = -0.001 * C;
    uint8_t success = 0;
    if (st->n_obj > 0) {
      const double d = dist3(tip, st->obj[0]), e = dist3(st->obj[0], st->goal);
      const int pick = event == 1 && st->held == 0;
      if (a[10] >= 0.5 && st->held != 0) {
        if (fabs(e - 0.15) < ORC_BAND) nb++;
        success = e < 0.15;
      }
      r += 10.0 * success + 5.0 * pick + (st->prev_d - d) + (st->prev_e - e);
      st->prev_d = d;
      st->prev_e = e;
    }
    for (int k = 0; k < 7; ++k) st->prev_a[k] = a[2 + k];
    const double c = cos(st->base[2]), sn = sin(st->base[2]);
    const double pb[3] = {st->base[0], 0.0, st->base[1]};
    const double* from[4] = {pb, pb, tip, tip};
    const double* to[4] = {st->obj_start, st->goal, st->obj_start, st->goal};
    for (int v = 0; v < 4; ++v) {
      const double w[3] = {to[v][0] - from[v][0], to[v][1] - from[v][1], to[v][2] - from[v][2]};
      out->task_obs[3 * v] = c * w[0] - sn * w[2];
      out->task_obs[3 * v + 1] = w[1];
      out->task_obs[3 * v + 2] = sn * w[0] + c * w[2];
    }
    out->reward = r;
    out->success = success;
  }

  *nbp += nb;
}

/* One step with the oriented-box object model (st->boxes): robot spheres
 * against the static grid and the resting boxes (exact sphere-box distance
 * in the box frame); a held box as its eight spheres against the static
 * grid and the other boxes; grasp of the box nearest the tip sphere (by the
 * exact distance); release: the box turns upright about its current
 * heading, its four bottom spheres are cast down and it rests on the
 * highest of their landing heights, unless a cast finds no surface or it
 * would overlap another box (then it goes back to its pre-grasp pose). */
static void step_boxes(const orc_robot* rb, const orc_scene* sc, orc_state* st, const double a[11],
                       orc_step_out* out) {
  int nb = 0;
  double cb[3], cq[7];
  candidate_pose(rb, st, a, cb, cq);
  double links[8][12], ee[12], cam[12];
  double cs[ORC_MAX_SPHERES][3];
  orc_fk(rb, cb, cq, links, ee, NULL);
  for (int i = 0; i < rb->n_spheres; ++i) {
    double p[3] = {rb->sphere_pos[3 * i], rb->sphere_pos[3 * i + 1], rb->sphere_pos[3 * i + 2]};
    fr_apply(links[rb->sphere_link[i]], p, cs[i]);
  }
  uint32_t mask = 0;
  uint8_t flags = 0;
  const int h = st->held;
  for (int i = 0; i < rb->n_spheres; ++i) {
    const double r = rb->sphere_radius[i];
    if (static_contact(sc, cs[i], r, &nb)) { mask |= 1u << i; flags |= 1; }
    for (int j = 0; j < st->n_obj; ++j)
      if (j != h && sphere_box_contact(st, j, cs[i], r, &nb)) { mask |= 1u << i; flags |= 2; }
  }
  if (h >= 0) {
    /* the carried spheres at the candidate tool frame: c = T_ee (c_off + R_off k) */
    double loc[8][3];
    const double s = orc_box_spheres(st->box[h], loc);
    for (int k = 0; k < 8; ++k) {
      double o[3];
      for (int r = 0; r < 3; ++r)
        o[r] = st->c_off[r] + st->r_off[3 * r] * loc[k][0] + st->r_off[3 * r + 1] * loc[k][1] +
               st->r_off[3 * r + 2] * loc[k][2];
      double c[3];
      fr_apply(ee, o, c);
      if (static_contact(sc, c, s, &nb)) { mask |= 1u << 30; flags |= 1 | 4; }
      for (int j = 0; j < st->n_obj; ++j)
        if (j != h && sphere_box_contact(st, j, c, s, &nb)) { mask |= 1u << 30; flags |= 2 | 4; }
    }
  }
  const int reverted = mask != 0;
  if (!reverted) {
    memcpy(st->base, cb, sizeof(cb));
    memcpy(st->q, cq, sizeof(cq));
  }
  orc_fk(rb, st->base, st->q, links, ee, cam);

  uint8_t event = 0;
  const int grasp = a[9] >= 0.5;
  if (grasp && st->held < 0) {
    const double tip[3] = {ee[9], ee[10], ee[11]};
    const double rg = rb->grasp_radius;
    int best = -1;
    double bests = INFINITY;
    for (int j = 0; j < st->n_obj; ++j) {
      const double d = orc_box_distance(st, j, tip);
      if (fabs(d - rg) < ORC_BAND) nb++;
      if (d < rg) {
        if (best >= 0 && fabs(d - bests) < ORC_BAND) nb++;
        if (d < bests) { bests = d; best = j; }
      }
    }
    if (best >= 0) {
      /* c_off = R_ee^T (p - t_ee), R_off = R_ee^T R_y(yaw) */
      const double* p = st->obj[best];
      const double dp[3] = {p[0] - ee[9], p[1] - ee[10], p[2] - ee[11]};
      double Ry[9];
      box_rotation(st, best, ee, Ry);  /* not yet held: R_y(yaw) */
      for (int r = 0; r < 3; ++r) {
        st->c_off[r] = ee[r] * dp[0] + ee[3 + r] * dp[1] + ee[6 + r] * dp[2];
        for (int c = 0; c < 3; ++c)
          st->r_off[3 * r + c] = ee[r] * Ry[c] + ee[3 + r] * Ry[3 + c] + ee[6 + r] * Ry[6 + c];
      }
      memcpy(st->p_pre, p, 3 * sizeof(double));
      st->held = best;
      event = 1;
    } else {
      event = 2;
    }
  } else if (!grasp && st->held >= 0) {
    const int j = st->held;
    double p[3], R[9];
    fr_apply(ee, st->c_off, p);
    box_rotation(st, j, ee, R);
    const double yaw = upright_yaw(R, &nb);
    const double* hb = st->box[j];
    double loc[8][3];
    const double s = orc_box_spheres(hb, loc);
    const double cy = cos(yaw), sy = sin(yaw);
    int ok = 1;
    double ytop = -INFINITY;
    for (int k = 0; k < 8; ++k) {
      if ((k >> 1) & 1) continue;  /* the four bottom spheres */
      const double b[3] = {p[0] + cy * loc[k][0] + sy * loc[k][2], p[1] + loc[k][1],
                           p[2] - sy * loc[k][0] + cy * loc[k][2]};
      int okk = 0;
      const double y = orc_snap(sc, b, s + (double)rb->rest_clearance, &okk, &nb);
      ok &= okk;
      if (y > ytop) ytop = y;
    }
    const double land[3] = {p[0], ytop + (hb[1] - s), p[2]};
    const double bl[4] = {hb[0], hb[1], hb[2], yaw};
    int overlap = 0;
    if (ok)
      for (int m = 0; m < st->n_obj; ++m)
        if (m != j && orc_boxes_overlap(land, bl, st->obj[m], st->box[m], &nb)) overlap = 1;
    if (ok && !overlap) {
      memcpy(st->obj[j], land, sizeof(land));
      st->box[j][3] = yaw;
      event = 3;
    } else {
      memcpy(st->obj[j], st->p_pre, 3 * sizeof(double));
      event = 4;
    }
    st->held = -1;
    memset(st->c_off, 0, sizeof(st->c_off));
    memset(st->r_off, 0, sizeof(st->r_off));
  }
  if (st->held >= 0) fr_apply(ee, st->c_off, st->obj[st->held]);
  st->step_count += 1;
  task_epilogue(st, a, ee, event, out, &nb);
  out->contact_mask = mask;
  out->flags = flags;
  out->event = event;
  out->reverted = (uint8_t)reverted;
  out->near_band = nb;
  out->ee[0] = ee[9]; out->ee[1] = ee[10]; out->ee[2] = ee[11];
  memcpy(out->cam_R, cam, 9 * sizeof(double));
  memcpy(out->cam_t, cam + 9, 3 * sizeof(double));
}

void orc_step_ex(const orc_robot* rb, const orc_scene* sc, orc_state* st, const float act[11],
                 const orc_step_opts* opt, orc_step_out* out) {
  if (st->boxes) {  /* the oriented-box object model: the plain step only */
    double ab[11];
    clip_actions(act, ab);
    step_boxes(rb, sc, st, ab, out);
    return;
  }
  const double* dhat = opt->dhat;
  const double margin = opt->margin, band = opt->band;
  double a[11];
  clip_actions(act, a);
  int nb = 0;

  double cb[3], cq[7];
  candidate_pose(rb, st, a, cb, cq);

  /* candidate spheres */
  double links[8][12], ee[12], cam[12];
  double cs[ORC_MAX_SPHERES][3];
  orc_fk(rb, cb, cq, links, ee, NULL);
  for (int i = 0; i < rb->n_spheres; ++i) {
    double p[3] = {rb->sphere_pos[3 * i], rb->sphere_pos[3 * i + 1], rb->sphere_pos[3 * i + 2]};
    fr_apply(links[rb->sphere_link[i]], p, cs[i]);
  }
  uint32_t mask = 0;
  uint8_t flags = 0;
  int h = st->held;
  for (int i = 0; i < rb->n_spheres; ++i) {
    double r = rb->sphere_radius[i];
    int hit = opt->column ? orc_column_contact(sc, cs[i], r, &nb)
              : dhat      ? neural_static_contact(sc, cs[i], r, dhat[i], margin, band, &nb)
                          : static_contact(sc, cs[i], r, &nb);
    if (hit) { mask |= 1u << i; flags |= 1; }
    for (int j = 0; j < st->n_obj; ++j) {
      if (j == h) continue;
      if (pair_contact(cs[i], r, st->obj[j], st->obj[j][3], &nb)) { mask |= 1u << i; flags |= 2; }
    }
  }
  if (h >= 0) {
    double ph[3];
    fr_apply(ee, st->c_off, ph);
    double rho = st->obj[h][3];
    int hit = opt->column ? orc_column_contact(sc, ph, rho, &nb)
              : dhat      ? neural_static_contact(sc, ph, rho, dhat[30], margin, band, &nb)
                          : static_contact(sc, ph, rho, &nb);
    if (hit) { mask |= 1u << 30; flags |= 1 | 4; }
    for (int j = 0; j < st->n_obj; ++j) {
      if (j == h) continue;
      if (pair_contact(ph, rho, st->obj[j], st->obj[j][3], &nb)) { mask |= 1u << 30; flags |= 2 | 4; }
    }
  }
  /* resolution: any contact rejects all robot motion for this step, unless
   * sliding finds a contact-free base position nearby */
  int reverted = mask != 0;
  if (reverted && opt->slide) {
    double ph[3] = {0, 0, 0}, off[2];
    if (h >= 0) fr_apply(ee, st->c_off, ph);
    if (slide_search(rb, sc, st, cs, ph, off, &nb)) {
      cb[0] += off[0];
      cb[1] += off[1];
      reverted = 0;
      flags |= 8;
    }
  }
  if (!reverted) {
    memcpy(st->base, cb, sizeof(cb));
    memcpy(st->q, cq, sizeof(cq));
  }
  orc_fk(rb, st->base, st->q, links, ee, cam);

  /* grasp / release at the accepted pose */
  uint8_t event = 0;
  int grasp = a[9] >= 0.5;
  if (grasp && st->held < 0) {
    double tip[3] = {ee[9], ee[10], ee[11]};
    double rg = rb->grasp_radius;
    int best = -1;
    double bests = INFINITY;
    for (int j = 0; j < st->n_obj; ++j) {
      double d = dist3(tip, st->obj[j]);
      if (fabs(d - (rg + st->obj[j][3])) < ORC_BAND) nb++;
      if (d < rg + st->obj[j][3]) {
        double sdist = d - st->obj[j][3];
        if (best >= 0 && fabs(sdist - bests) < ORC_BAND) nb++;
        if (sdist < bests) { bests = sdist; best = j; }
      }
    }
    if (best >= 0) {
      /* c_off = R_ee^T (p - t_ee) */
      double dp[3] = {st->obj[best][0] - ee[9], st->obj[best][1] - ee[10], st->obj[best][2] - ee[11]};
      for (int r = 0; r < 3; ++r) st->c_off[r] = ee[r] * dp[0] + ee[3 + r] * dp[1] + ee[6 + r] * dp[2];
      memcpy(st->p_pre, st->obj[best], 3 * sizeof(double));
      st->held = best;
      event = 1;
    } else {
      event = 2;
    }
  } else if (!grasp && st->held >= 0) {
    int j = st->held;
    double p[3];
    fr_apply(ee, st->c_off, p);
    double rho = st->obj[j][3];
    int ok = 0;
    double y = orc_snap(sc, p, rho + (double)rb->rest_clearance, &ok, &nb);
    double land[3] = {p[0], y, p[2]};
    int overlap = 0;
    if (ok)
      for (int k = 0; k < st->n_obj; ++k)
        if (k != j && pair_contact(land, rho, st->obj[k], st->obj[k][3], &nb)) overlap = 1;
    int jittered = 0;
    if (!(ok && !overlap) && opt->place_jitter) {
      /* Object placing heuristic (appendix "Object Placing Heuristic"): at
       * most six jitters of 2 rho in the ground plane, each followed by a new
       * cast down from the release height.  Direction: away from the
       * objects the landing overlaps (sum of unit ground-plane vectors),
       * turned by a uniform angle in [-pi/4, pi/4); a uniform direction when
       * nothing overlaps.  Draw k: Philox4x32-10 on (env, step, k,
       * 0x4A495454) with the reset key. */
      const uint32_t key[2] = {(uint32_t)opt->seed, (uint32_t)(opt->seed >> 32)};
      double q[3] = {land[0], land[1], land[2]};
      int landed = ok;  /* the current trial position rests on a surface */
      for (uint32_t k = 0; k < 6 && !jittered; ++k) {
        double Dx = 0.0, Dz = 0.0;
        if (landed)
          for (int m = 0; m < st->n_obj; ++m) {
            if (m == j) continue;
            if (dist3(q, st->obj[m]) < rho + st->obj[m][3]) {
              double vx = q[0] - st->obj[m][0], vz = q[2] - st->obj[m][2];
              double vl = sqrt(vx * vx + vz * vz);
              if (vl > 1e-9) { Dx += vx / vl; Dz += vz / vl; }
            }
          }
        uint32_t ctr[4] = {(uint32_t)opt->env, (uint32_t)st->step_count, k, 0x4A495454u}, w[4];
        orc_philox4x32_10(ctr, key, w);
        double u = unit24(w[0]), dl = sqrt(Dx * Dx + Dz * Dz), phi;
        if (dl > 1e-6) {
          if (dl < 1e-4) nb++;
          phi = atan2(Dz, Dx) + (u - 0.5) * (PI / 2);
        } else {
          phi = 2 * PI * u;
        }
        q[0] += 2 * rho * cos(phi);
        q[2] += 2 * rho * sin(phi);
        double cast[3] = {q[0], p[1], q[2]};
        int ok2 = 0;
        double y2 = orc_snap(sc, cast, rho + (double)rb->rest_clearance, &ok2, &nb);
        q[1] = ok2 ? y2 : p[1];
        landed = ok2;
        int ov2 = 0;
        if (ok2)
          for (int m = 0; m < st->n_obj; ++m)
            if (m != j && pair_contact(q, rho, st->obj[m], st->obj[m][3], &nb)) ov2 = 1;
        if (ok2 && !ov2) {
          memcpy(land, q, sizeof(land));
          jittered = 1;
        }
      }
    }
    if (ok && !overlap) {
      memcpy(st->obj[j], land, sizeof(land));
      event = 3;
    } else if (jittered) {
      memcpy(st->obj[j], land, sizeof(land));
      event = 5;
    } else {
      memcpy(st->obj[j], st->p_pre, 3 * sizeof(double));
      event = 4;
    }
    st->held = -1;
    memset(st->c_off, 0, sizeof(st->c_off));
  }
  if (st->held >= 0) fr_apply(ee, st->c_off, st->obj[st->held]);
  st->step_count += 1;

  task_epilogue(st, a, ee, event, out, &nb);

  out->contact_mask = mask;
  out->flags = flags;
  out->event = event;
  out->reverted = (uint8_t)reverted;
  out->near_band = nb;
  out->ee[0] = ee[9]; out->ee[1] = ee[10]; out->ee[2] = ee[11];
  memcpy(out->cam_R, cam, 9 * sizeof(double));
  memcpy(out->cam_t, cam + 9, 3 * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* Reset: objects on support tops, then the robot base in free space, each  */
/* by rejection sampling with at most 64 Philox draws.  Stream (env,        */
/* episode, j, try): j = object index, ORC_MAX_OBJ = robot, ORC_MAX_OBJ + 1 */
/* = the task's goal.                                                       */
/* ------------------------------------------------------------------------ */
void orc_reset(const orc_robot* rb, const orc_scene* sc, orc_state* st, uint64_t seed,
               int32_t env, int32_t n_obj, float rho_min, float rho_max, orc_reset_out* out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int nb = 0, failed = 0;
  st->episode += 1;
  st->n_obj = n_obj;
  double clear = rb->rest_clearance;
  for (int j = 0; j < n_obj && st->boxes; ++j) {
    /* oriented boxes: half extents from one draw per object (counter word 3
     * = 0x424F5845), each try a support, a position on its top shrunk by
     * the footprint's circumradius, and a yaw; accepted when the box's
     * eight spheres are clear of the static scene and it overlaps no box
     * placed before it */
    uint32_t cs0[4] = {(uint32_t)env, (uint32_t)st->episode, (uint32_t)j, 0x424F5845u}, ws[4];
    orc_philox4x32_10(cs0, key, ws);
    double* hb = st->box[j];
    for (int a = 0; a < 3; ++a)
      hb[a] = (double)rho_min + unit24(ws[a]) * ((double)rho_max - (double)rho_min);
    const double rxz = sqrt(hb[0] * hb[0] + hb[2] * hb[2]);
    double loc[8][3];
    const double sr = orc_box_spheres(hb, loc);
    int ok = 0;
    for (uint32_t t = 0; t < 64 && !ok; ++t) {
      uint32_t ctr[4] = {(uint32_t)env, (uint32_t)st->episode, (uint32_t)j, t}, w[4];
      orc_philox4x32_10(ctr, key, w);
      uint32_t si = (uint32_t)(((uint64_t)(w[0] >> 8) * (uint64_t)sc->n_supports) >> 24);
      const float* sp = sc->supports + 5 * si;
      double x0 = sp[0] + rxz, x1 = sp[2] - rxz, z0 = sp[1] + rxz, z1 = sp[3] - rxz;
      double p[3] = {x0 + unit24(w[1]) * (x1 - x0), (double)sp[4] + hb[1] + clear,
                     z0 + unit24(w[2]) * (z1 - z0)};
      hb[3] = -PI + unit24(w[3]) * (2 * PI);
      st->obj[j][0] = p[0]; st->obj[j][1] = p[1]; st->obj[j][2] = p[2];
      st->obj[j][3] = sqrt(hb[0] * hb[0] + hb[1] * hb[1] + hb[2] * hb[2]);
      const double cy = cos(hb[3]), sy = sin(hb[3]);
      ok = 1;
      for (int k = 0; k < 8 && ok; ++k) {
        const double c[3] = {p[0] + cy * loc[k][0] + sy * loc[k][2], p[1] + loc[k][1],
                             p[2] - sy * loc[k][0] + cy * loc[k][2]};
        if (static_contact(sc, c, sr, &nb)) ok = 0;
      }
      for (int k = 0; k < j && ok; ++k)
        if (orc_boxes_overlap(p, hb, st->obj[k], st->box[k], &nb)) ok = 0;
    }
    if (!ok) failed++;
  }
  for (int j = 0; j < n_obj && !st->boxes; ++j) {
    double rho = 0.0;
    int ok = 0;
    for (uint32_t t = 0; t < 64 && !ok; ++t) {
      uint32_t ctr[4] = {(uint32_t)env, (uint32_t)st->episode, (uint32_t)j, t}, w[4];
      orc_philox4x32_10(ctr, key, w);
      if (t == 0) rho = (double)rho_min + unit24(w[3]) * ((double)rho_max - (double)rho_min);
      uint32_t si = (uint32_t)(((uint64_t)(w[0] >> 8) * (uint64_t)sc->n_supports) >> 24);
      const float* sp = sc->supports + 5 * si;
      double x0 = sp[0] + rho, x1 = sp[2] - rho, z0 = sp[1] + rho, z1 = sp[3] - rho;
      double p[3] = {x0 + unit24(w[1]) * (x1 - x0), (double)sp[4] + rho + clear,
                     z0 + unit24(w[2]) * (z1 - z0)};
      st->obj[j][0] = p[0]; st->obj[j][1] = p[1]; st->obj[j][2] = p[2]; st->obj[j][3] = rho;
      ok = !static_contact(sc, p, rho, &nb);
      for (int k = 0; k < j && ok; ++k)
        if (pair_contact(p, rho, st->obj[k], st->obj[k][3], &nb)) ok = 0;
    }
    if (!ok) failed++;
  }
  double cs[ORC_MAX_SPHERES][3];
  int ok = 0;
  for (int k = 0; k < 7; ++k) st->q[k] = rb->q_rest[k];
  for (uint32_t t = 0; t < 64 && !ok; ++t) {
    uint32_t ctr[4] = {(uint32_t)env, (uint32_t)st->episode, ORC_MAX_OBJ, t}, w[4];
    orc_philox4x32_10(ctr, key, w);
    const float* s = sc->spawn;
    st->base[0] = s[0] + unit24(w[0]) * ((double)s[2] - (double)s[0]);
    st->base[1] = s[1] + unit24(w[1]) * ((double)s[3] - (double)s[1]);
    st->base[2] = -PI + unit24(w[2]) * (2 * PI);
    orc_sphere_centres(rb, st->base, st->q, cs);
    ok = 1;
    for (int i = 0; i < rb->n_spheres; ++i) {
      double r = rb->sphere_radius[i];
      int c = static_contact(sc, cs[i], r, &nb);
      for (int j = 0; j < n_obj; ++j)
        c |= st->boxes ? sphere_box_contact(st, j, cs[i], r, &nb)
                       : pair_contact(cs[i], r, st->obj[j], st->obj[j][3], &nb);
      if (c) ok = 0;
    }
  }
  if (!ok) failed++;
  st->held = -1;
  memset(st->c_off, 0, sizeof(st->c_off));
  memset(st->p_pre, 0, sizeof(st->p_pre));
  memset(st->r_off, 0, sizeof(st->r_off));
  st->step_count = 0;
  /* task: object 0 is the target; its goal lies on a support top, drawn
   * like an object placement from stream ORC_MAX_OBJ + 1 (first draw, not tested for
   * collisions); the previous distances start at the episode's first pose
   * and the previous joint actions at 0. */
  memset(st->goal, 0, sizeof(st->goal));
  memset(st->obj_start, 0, sizeof(st->obj_start));
  memset(st->prev_a, 0, sizeof(st->prev_a));
  st->prev_d = st->prev_e = 0.0;
  if (n_obj > 0 && sc->n_supports > 0) {
    uint32_t ctr[4] = {(uint32_t)env, (uint32_t)st->episode, ORC_MAX_OBJ + 1, 0u}, w[4];
    orc_philox4x32_10(ctr, key, w);
    /* a box target: shrunk by its footprint's circumradius, raised by hy */
    const double rho = st->boxes ? sqrt(st->box[0][0] * st->box[0][0] + st->box[0][2] * st->box[0][2])
                                 : st->obj[0][3];
    const double lift = st->boxes ? st->box[0][1] : st->obj[0][3];
    uint32_t si = (uint32_t)(((uint64_t)(w[0] >> 8) * (uint64_t)sc->n_supports) >> 24);
    const float* sp = sc->supports + 5 * si;
    double x0 = sp[0] + rho, x1 = sp[2] - rho, z0 = sp[1] + rho, z1 = sp[3] - rho;
    st->goal[0] = x0 + unit24(w[1]) * (x1 - x0);
    st->goal[1] = (double)sp[4] + lift + clear;
    st->goal[2] = z0 + unit24(w[2]) * (z1 - z0);
    memcpy(st->obj_start, st->obj[0], 3 * sizeof(double));
    double links[8][12], ee[12];
    orc_fk(rb, st->base, st->q, links, ee, NULL);
    const double tip[3] = {ee[9], ee[10], ee[11]};
    st->prev_d = dist3(tip, st->obj[0]);
    st->prev_e = dist3(st->obj[0], st->goal);
  }
  out->near_band = nb;
  out->failed = failed;
}

/* ------------------------------------------------------------------------ */
/* Rendering (Sec. 3.1): for every pixel centre, the nearest front-facing   */
/* triangle hit by the camera ray at planar depth z >= near.  Depth is the  */
/* camera-space forward distance of the hit, colour that triangle's flat    */
/* colour; no hit gives 0 / black.  The result is the minimum over          */
/* triangles, so it does not depend on visiting order: each triangle only   */
/* evaluates pixel centres inside its projected bounding box (grown by one  */
/* pixel), the only ones it can cover.                                      */
/*                                                                          */
/* Alongside the exact answer each pixel gets an "ambiguous" bit: true when */
/* an FP32 fixed-point rasteriser could legitimately produce a different    */
/* visible surface there -- a pixel centre within eps_px of an edge of a    */
/* triangle that competes for the pixel, two surfaces within tol_rel in     */
/* depth with different colours, or a grazing hit (|cos| < cos_min).        */
/* ------------------------------------------------------------------------ */
#define ORC_K 16
typedef struct { double z, s, cosv; int32_t id; uint32_t rgb; } cand;

static int clip_near(const double in[3][3], double near, double out[4][3]) {
  int n = 0;
  for (int k = 0; k < 3; ++k) {
    const double* a = in[k];
    const double* b = in[(k + 1) % 3];
    int ain = a[2] >= near, bin = b[2] >= near;
    if (ain) { memcpy(out[n++], a, 3 * sizeof(double)); }
    if (ain != bin) {
      double t = (near - a[2]) / (b[2] - a[2]);
      out[n][0] = a[0] + t * (b[0] - a[0]);
      out[n][1] = a[1] + t * (b[1] - a[1]);
      out[n][2] = near;
      n++;
    }
  }
  return n;
}

static void render_tri(const double P[3][3], int32_t id, uint32_t col, const double cam[12],
                       double near, int W, int H, double eps, cand* C, int* cnt, double* dropz,
                       orc_render_stats* stats) {
  const double* eye = cam + 9;
  double e1[3], e2[3], n[3];
  for (int a = 0; a < 3; ++a) { e1[a] = P[1][a] - P[0][a]; e2[a] = P[2][a] - P[0][a]; }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  double hpl = n[0] * (P[0][0] - eye[0]) + n[1] * (P[0][1] - eye[1]) + n[2] * (P[0][2] - eye[2]);
  if (!(hpl < 0)) return; /* back-facing or edge-on */
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  /* camera-space vertices: columns of R are right, up, forward */
  double Cv[3][3];
  for (int k = 0; k < 3; ++k) {
    double d[3] = {P[k][0] - eye[0], P[k][1] - eye[1], P[k][2] - eye[2]};
    for (int c = 0; c < 3; ++c) Cv[k][c] = cam[c] * d[0] + cam[3 + c] * d[1] + cam[6 + c] * d[2];
  }
  double poly[4][3], uv[4][2];
  int m = clip_near(Cv, near, poly);
  if (m < 3) return;
  double f = 0.5 * W, cx = 0.5 * W, cy = 0.5 * H;
  double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
  for (int k = 0; k < m; ++k) {
    uv[k][0] = cx + f * poly[k][0] / poly[k][2];
    uv[k][1] = cy - f * poly[k][1] / poly[k][2];
    umin = fmin(umin, uv[k][0]); umax = fmax(umax, uv[k][0]);
    vmin = fmin(vmin, uv[k][1]); vmax = fmax(vmax, uv[k][1]);
  }
  double area2 = 0.0;
  for (int k = 0; k < m; ++k) {
    int l = (k + 1) % m;
    area2 += uv[k][0] * uv[l][1] - uv[l][0] * uv[k][1];
  }
  if (area2 == 0.0) return;
  double sgn = area2 > 0 ? 1.0 : -1.0;
  int i0 = (int)floor(umin - 1.0), i1 = (int)ceil(umax + 1.0);
  int j0 = (int)floor(vmin - 1.0), j1 = (int)ceil(vmax + 1.0);
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  if (i1 > W - 1) i1 = W - 1;
  if (j1 > H - 1) j1 = H - 1;
  if (i0 > i1 || j0 > j1) return;
  /* a triangle counts as set up when some pixel centre lies in its bounding box */
  if (ceil(umin - 0.5) <= fmin(floor(umax - 0.5), W - 1.0) && ceil(umax - 0.5) >= 0.0 &&
      ceil(vmin - 0.5) <= fmin(floor(vmax - 0.5), H - 1.0) && ceil(vmax - 0.5) >= 0.0 &&
      floor(umax - 0.5) >= 0.0 && floor(vmax - 0.5) >= 0.0)
    stats->tris_setup++;
  double len[4];
  for (int k = 0; k < m; ++k) {
    int l = (k + 1) % m;
    len[k] = hypot(uv[l][0] - uv[k][0], uv[l][1] - uv[k][1]);
  }
  for (int j = j0; j <= j1; ++j)
    for (int i = i0; i <= i1; ++i) {
      double u = i + 0.5, v = j + 0.5;
      double s = INFINITY;
      for (int k = 0; k < m; ++k) {
        int l = (k + 1) % m;
        if (len[k] == 0.0) continue;
        double e = (uv[l][0] - uv[k][0]) * (v - uv[k][1]) - (uv[l][1] - uv[k][1]) * (u - uv[k][0]);
        double sd = sgn * e / len[k];
        if (sd < s) s = sd;
      }
      if (!(s > -eps)) continue;
      double dc[3] = {(u - cx) / f, -(v - cy) / f, 1.0};
      double D[3];
      for (int r = 0; r < 3; ++r) D[r] = cam[3 * r] * dc[0] + cam[3 * r + 1] * dc[1] + cam[3 * r + 2] * dc[2];
      double nd = n[0] * D[0] + n[1] * D[1] + n[2] * D[2];
      if (!(nd < 0)) continue;
      double z = hpl / nd;
      double dl = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
      if (s > 0) stats->frags_covered++;
      cand c = {z, s, -nd / (nn * dl), id, col};
      cand* L = C + (size_t)(j * W + i) * ORC_K;
      int* nc = cnt + j * W + i;
      /* keep the ORC_K nearest, sorted by z then id */
      int pos = *nc;
      while (pos > 0 && (L[pos - 1].z > z || (L[pos - 1].z == z && L[pos - 1].id > id))) pos--;
      if (pos >= ORC_K) {
        if (z < dropz[j * W + i]) dropz[j * W + i] = z;
        continue;
      }
      if (*nc == ORC_K) {
        double zl = L[ORC_K - 1].z;
        if (zl < dropz[j * W + i]) dropz[j * W + i] = zl;
      } else {
        (*nc)++;
      }
      for (int q = *nc - 1; q > pos; --q) L[q] = L[q - 1];
      L[pos] = c;
    }
}

void orc_render(const orc_robot* rb, const orc_scene* sc, const orc_objmesh* om,
                const orc_state* st, int32_t W, int32_t H, double eps_px, double tol_rel,
                double cos_min, double* depth, uint32_t* rgb, uint8_t* ambiguous,
                int32_t* winner, orc_render_stats* stats) {
  orc_render_cos(rb, sc, om, st, W, H, eps_px, tol_rel, cos_min, depth, rgb, ambiguous, winner,
                 stats, NULL);
}

void orc_render_cos(const orc_robot* rb, const orc_scene* sc, const orc_objmesh* om,
                    const orc_state* st, int32_t W, int32_t H, double eps_px, double tol_rel,
                    double cos_min, double* depth, uint32_t* rgb, uint8_t* ambiguous,
                    int32_t* winner, orc_render_stats* stats, double* cos_out) {
  double links[8][12], cam[12];
  orc_fk(rb, st->base, st->q, links, NULL, cam);
  size_t np = (size_t)W * H;
  cand* C = (cand*)malloc(np * ORC_K * sizeof(cand));
  int* cnt = (int*)calloc(np, sizeof(int));
  double* dropz = (double*)malloc(np * sizeof(double));
  for (size_t p = 0; p < np; ++p) dropz[p] = INFINITY;
  orc_render_stats local = {0, 0, 0, 0};
  double near = rb->cam_near;
  double P[3][3];
  for (int t = 0; t < sc->n_tris; ++t) {
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 3; ++a) P[k][a] = sc->verts[3 * sc->tris[3 * t + k] + a];
    render_tri(P, t, sc->tri_rgb[t], cam, near, W, H, eps_px, C, cnt, dropz, &local);
  }
  double ee[12];
  if (st->boxes) orc_fk(rb, st->base, st->q, links, ee, NULL);
  for (int j = 0; j < st->n_obj; ++j) {
    /* a sphere: the mesh scaled by rho; a box: the unit cube mesh mapped by
     * R diag(h), R its world rotation */
    double M[9] = {st->obj[j][3], 0, 0, 0, st->obj[j][3], 0, 0, 0, st->obj[j][3]};
    if (st->boxes) {
      double R[9];
      box_rotation(st, j, ee, R);
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * st->box[j][c];
    }
    for (int t = 0; t < om->n_tris; ++t) {
      for (int k = 0; k < 3; ++k) {
        const float* u = om->verts + 3 * om->tris[3 * t + k];
        for (int a = 0; a < 3; ++a)
          P[k][a] = st->obj[j][a] + M[3 * a] * (double)u[0] + M[3 * a + 1] * (double)u[1] +
                    M[3 * a + 2] * (double)u[2];
      }
      render_tri(P, sc->n_tris + j * om->n_tris + t, om->obj_rgb[j], cam, near, W, H, eps_px, C,
                 cnt, dropz, &local);
    }
  }
  /* the robot body: its collision spheres as the same instanced mesh, in
   * instance slots ORC_MAX_OBJ + i */
  if (om->robot_rgb) {
    double cs[ORC_MAX_SPHERES][3];
    orc_sphere_centres(rb, st->base, st->q, cs);
    for (int i = 0; i < rb->n_spheres; ++i) {
      const double r = rb->sphere_radius[i];
      for (int t = 0; t < om->n_tris; ++t) {
        for (int k = 0; k < 3; ++k)
          for (int a = 0; a < 3; ++a)
            P[k][a] = cs[i][a] + r * (double)om->verts[3 * om->tris[3 * t + k] + a];
        render_tri(P, sc->n_tris + (ORC_MAX_OBJ + i) * om->n_tris + t, om->robot_rgb[i], cam,
                   near, W, H, eps_px, C, cnt, dropz, &local);
      }
    }
  }
  for (size_t p = 0; p < np; ++p) {
    cand* L = C + p * ORC_K;
    int nc = cnt[p];
    int w = -1;
    double zD = INFINITY;
    for (int q = 0; q < nc; ++q) {
      if (w < 0 && L[q].s > 0) w = q;
      if (L[q].s > eps_px && L[q].z < zD) zD = L[q].z;
    }
    uint8_t amb = 0;
    double zw = w >= 0 ? L[w].z : INFINITY;
    if (dropz[p] <= zD * (1 + tol_rel)) { amb = 1; local.overflow++; }
    for (int q = 0; q < nc; ++q) {
      if (!(L[q].z <= zD * (1 + tol_rel))) continue; /* loses the depth test */
      if (w < 0) { amb = 1; break; }                  /* marginal vs background */
      if (L[q].rgb != L[w].rgb || fabs(L[q].z - zw) > tol_rel * zw) { amb = 1; break; }
    }
    if (w >= 0 && L[w].cosv < cos_min) amb = 1;
    depth[p] = w >= 0 ? zw : 0.0;
    rgb[p] = w >= 0 ? L[w].rgb : 0u;
    if (winner) winner[p] = w >= 0 ? L[w].id : -1;
    if (cos_out) cos_out[p] = w >= 0 ? L[w].cosv : 1.0;
    ambiguous[p] = amb;
    local.ambiguous += amb;
  }
  if (stats) *stats = local;
  free(C);
  free(cnt);
  free(dropz);
}

/* ------------------------------------------------------------------------ */
/* Neural-SDF training sample i (the workload's learned part; not in the     */
/* paper).  Even i: one uniform draw over the lattice box.  Odd i: the first */
/* of at most 64 uniform draws whose interpolated distance has |d| < band,   */
/* or the last draw when none has.  Draw t of sample i takes Philox4x32-10  */
/* on counter (i, scene, t, 0x4E534446) with key (seed low, seed high);     */
/* coordinate a = origin_a + u_a (dims_a - 1) h with u_a = (word_a >> 8) /  */
/* 2^24.  The label is the trilinear grid distance at the drawn point.       */
/* Returns the index of the draw used; *near_band counts draws whose |d|    */
/* lay within ORC_BAND of band.                                              */
/* ------------------------------------------------------------------------ */
int orc_nsdf_sample(const orc_scene* s, uint64_t seed, uint32_t scene, uint32_t i, double band,
                    double p[3], double* d, int* near_band) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const int tries = (i & 1u) ? 64 : 1;
  int nb = 0, t = 0;
  for (t = 0; t < tries; ++t) {
    uint32_t ctr[4] = {i, scene, (uint32_t)t, 0x4E534446u}, w[4];
    orc_philox4x32_10(ctr, key, w);
    for (int a = 0; a < 3; ++a)
      p[a] = (double)s->grid_origin[a] +
             unit24(w[a]) * ((double)(s->grid_dims[a] - 1) * (double)s->grid_h);
    double edge;
    orc_grid_query(s, p, d, &edge);
    if (tries == 1) break;
    if (fabs(fabs(*d) - band) < ORC_BAND) nb++;
    if (fabs(*d) < band) break;
  }
  if (near_band) *near_band = nb;
  return t < tries ? t : tries - 1;
}

/* ------------------------------------------------------------------------ */
/* Neural SDF: d(x) = W_L relu(... relu(W_1 gamma(x) + b_1) ...) + b_L with  */
/* Fourier features gamma(x) = [sin(2 pi B x), cos(2 pi B x)].              */
/* dims = {2F, h1, ..., 1}; W[l] is row-major [dims[l+1]][dims[l]].         */
/* ------------------------------------------------------------------------ */
/* Optional rounding of every GEMM operand the tensor-core kernels feed in
 * BF16 (features, hidden activations, back-propagated gradients), to the
 * nearest BF16 (ties to even) through float; the arithmetic stays FP64. */
static int g_mlp_bf16 = 0;
void orc_mlp_set_bf16_operands(int on) { g_mlp_bf16 = on; }
static double bf16r(double x) {
  if (!g_mlp_bf16) return x;
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

static void mlp_acts(const double* B, int F, const double* const* W, const double* const* b,
                     const int* dims, int L, const double x[3], double* A) {
  /* A holds layer inputs back to back: a_0 (2F), a_1, ..., a_L (1) */
  for (int k = 0; k < F; ++k) {
    double ph = 2 * PI * (B[3 * k] * x[0] + B[3 * k + 1] * x[1] + B[3 * k + 2] * x[2]);
    A[k] = bf16r(sin(ph));
    A[F + k] = bf16r(cos(ph));
  }
  double* in = A;
  for (int l = 0; l < L; ++l) {
    double* o = in + dims[l];
    for (int r = 0; r < dims[l + 1]; ++r) {
      double s = b[l][r];
      for (int c = 0; c < dims[l]; ++c) s += W[l][(size_t)r * dims[l] + c] * in[c];
      o[r] = (l < L - 1 && s < 0) ? 0.0 : s;
      if (l < L - 1) o[r] = bf16r(o[r]);
    }
    in = o;
  }
}

double orc_mlp_forward(const double* B, int F, const double* const* W, const double* const* b,
                       const int* dims, int L, const double x[3], double* acts) {
  int tot = 0;
  for (int l = 0; l <= L; ++l) tot += dims[l];
  double* A = acts ? acts : (double*)malloc(tot * sizeof(double));
  mlp_acts(B, F, W, b, dims, L, x, A);
  double y = A[tot - 1];
  if (!acts) free(A);
  return y;
}

/* Mean L1 loss against clamped labels and its exact gradient (backprop). */
double orc_mlp_loss_grad(const double* B, int F, const double* const* W, const double* const* b,
                         const int* dims, int L, const double* X, const double* y, int n,
                         double lo, double hi, double* const* gW, double* const* gb) {
  int tot = 0, maxw = 0;
  for (int l = 0; l <= L; ++l) { tot += dims[l]; if (dims[l] > maxw) maxw = dims[l]; }
  for (int l = 0; l < L; ++l) {
    memset(gW[l], 0, (size_t)dims[l] * dims[l + 1] * sizeof(double));
    memset(gb[l], 0, (size_t)dims[l + 1] * sizeof(double));
  }
  double* A = (double*)malloc(tot * sizeof(double));
  double* g = (double*)malloc(maxw * sizeof(double));
  double* g2 = (double*)malloc(maxw * sizeof(double));
  double loss = 0.0;
  for (int s = 0; s < n; ++s) {
    mlp_acts(B, F, W, b, dims, L, X + 3 * s, A);
    double pred = A[tot - 1];
    double t = clampd(y[s], lo, hi);
    loss += fabs(pred - t);
    g[0] = (pred > t ? 1.0 : (pred < t ? -1.0 : 0.0)) / n;
    /* walk layers backwards; offsets of a_l in A */
    int off[16];
    off[0] = 0;
    for (int l = 0; l < L; ++l) off[l + 1] = off[l] + dims[l];
    for (int l = L - 1; l >= 0; --l) {
      const double* in = A + off[l];
      const double* outv = A + off[l + 1];
      /* g is dLoss/d(pre-activation of layer l) once the ReLU mask is applied */
      if (l < L - 1)
        for (int r = 0; r < dims[l + 1]; ++r) g[r] = (outv[r] > 0) ? bf16r(g[r]) : 0.0;
      for (int r = 0; r < dims[l + 1]; ++r) {
        gb[l][r] += g[r];
        for (int c = 0; c < dims[l]; ++c) gW[l][(size_t)r * dims[l] + c] += g[r] * in[c];
      }
      if (l > 0) {
        for (int c = 0; c < dims[l]; ++c) {
          double acc = 0.0;
          for (int r = 0; r < dims[l + 1]; ++r) acc += W[l][(size_t)r * dims[l] + c] * g[r];
          g2[c] = acc;
        }
        memcpy(g, g2, dims[l] * sizeof(double));
      }
    }
  }
  free(A);
  free(g);
  free(g2);
  return loss / n;
}

/* ------------------------------------------------------------------------ */
/* Rounding-error bound of the BF16-operand network against the plain one.  */
/* The plain network is the FP64 MLP above with nothing rounded.  A kernel   */
/* that rounds each operand a_{l,i} fed to a product (features a_0, hidden  */
/* activations a_1 .. a_{L-1}) to BF16, sums in FP32 over K terms and has   */
/* features within feat_err of sin/cos, differs from it, to first order in  */
/* the rounding errors (Higham, "Accuracy and Stability of Numerical        */
/* Algorithms", 2nd ed., Sec. 3.1 for the sums; the output's sensitivity    */
/* to each operand is its gradient), by at most                             */
/*   u_b sum_{l,i} |g_{l,i}| |a_{l,i}|          BF16 operand rounding        */
/* + feat_err (1 + u_b) sum_i |g_{0,i}|         feature error                */
/* + sum_{l,r} |gz_{l,r}| (gam_K (|W_l| |a_{l-1}|)_r + u_f (|z_{l,r}| + |b_{l,r}|))  */
/*                                               FP32 sums and bias adds    */
/* with g_{l,i} = dd/da_{l,i}, gz_{l,r} = dd/dz_{l,r} (z = pre-activation),  */
/* u_b = 2^-8 (BF16: 8 significant bits, round to nearest), u_f = 2^-24,    */
/* gam_K = 2 K u_f (an FP32 sum of K products, with a factor 2 for the      */
/* accumulation order of the tensor cores).  g is taken through the plain   */
/* network's ReLU masks, and |g_{l,i}| is the sensitivity to a_{l,i} itself */
/* (not masked by unit i's own ReLU).  Returns the plain d(x); terms[0..2]  */
/* get the operand, feature and FP32 parts of the bound (their sum), and    */
/* terms[3] the standard deviation of the operand part when the rounding    */
/* errors are independent and uniform in +-u_b |a|:                         */
/*   u_b sqrt(sum (g a)^2 / 3)  (a typical error, not a bound).             */
/* ------------------------------------------------------------------------ */
double orc_mlp_rounding_bound(const double* B, int F, const double* const* W,
                              const double* const* b, const int* dims, int L, const double x[3],
                              double feat_err, double terms[4]) {
  const double ub = 1.0 / 256.0, uf = 1.0 / 16777216.0;
  int tot = 0, maxw = 0;
  for (int l = 0; l <= L; ++l) { tot += dims[l]; if (dims[l] > maxw) maxw = dims[l]; }
  int off[17];
  off[0] = 0;
  for (int l = 0; l < L && l < 16; ++l) off[l + 1] = off[l] + dims[l];
  double* A = (double*)malloc(tot * sizeof(double));  /* a_0 .. a_L (plain)      */
  double* Z = (double*)malloc(tot * sizeof(double));  /* z_l at a_l's offsets   */
  double* g = (double*)malloc(maxw * sizeof(double));  /* dd/da_l                */
  double* g2 = (double*)malloc(maxw * sizeof(double));
  /* plain forward, nothing rounded */
  for (int k = 0; k < F; ++k) {
    double ph = 2 * PI * (B[3 * k] * x[0] + B[3 * k + 1] * x[1] + B[3 * k + 2] * x[2]);
    A[k] = sin(ph);
    A[F + k] = cos(ph);
  }
  for (int l = 0; l < L; ++l) {
    const double* in = A + off[l];
    for (int r = 0; r < dims[l + 1]; ++r) {
      double s = b[l][r];
      for (int c = 0; c < dims[l]; ++c) s += W[l][(size_t)r * dims[l] + c] * in[c];
      Z[off[l + 1] + r] = s;
      A[off[l + 1] + r] = (l < L - 1 && s < 0) ? 0.0 : s;
    }
  }
  const double d = A[off[L]];
  /* backward: g = dd/da_l for l = L-1 .. 0, accumulating the bound */
  double t_op = 0.0, t_feat = 0.0, t_f32 = 0.0, t_sq = 0.0;
  g[0] = 1.0;  /* dd/dz_L = 1 (linear output) */
  for (int l = L - 1; l >= 0; --l) {
    /* g holds dd/dz_{l+1} (pre-activation of layer l's output, masked) */
    const double* in = A + off[l];
    const double gam = 2.0 * dims[l] * uf;
    for (int r = 0; r < dims[l + 1]; ++r) {
      double absdot = 0.0;
      for (int c = 0; c < dims[l]; ++c) absdot += fabs(W[l][(size_t)r * dims[l] + c] * in[c]);
      t_f32 += fabs(g[r]) * (gam * absdot + uf * (fabs(Z[off[l + 1] + r]) + fabs(b[l][r])));
    }
    for (int c = 0; c < dims[l]; ++c) {
      double acc = 0.0;
      for (int r = 0; r < dims[l + 1]; ++r) acc += W[l][(size_t)r * dims[l] + c] * g[r];
      g2[c] = acc;  /* dd/da_{l,c} */
      t_op += ub * fabs(acc) * fabs(in[c]);
      t_sq += acc * acc * in[c] * in[c];
      if (l == 0) t_feat += feat_err * (1.0 + ub) * fabs(acc);
    }
    if (l > 0)
      for (int c = 0; c < dims[l]; ++c) g[c] = Z[off[l] + c] > 0 ? g2[c] : 0.0;
  }
  free(A);
  free(Z);
  free(g);
  free(g2);
  terms[0] = t_op;
  terms[1] = t_feat;
  terms[2] = t_f32;
  terms[3] = ub * sqrt(t_sq / 3.0);
  return d;
}
