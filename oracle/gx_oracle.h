/*
 * gx_oracle.h -- plain, single-threaded FP64 CPU oracle for the batched
 * environment step of Galactic (arXiv 2306.07552, Sec. 3.2 and the appendix
 * "Additional Collision-Detection Details").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library.  It shares no code with the CUDA
 * path: it reads the same *inputs* (robot table, scene boxes and triangles,
 * actions) and recomputes every step of the method from its definition, in
 * double precision, one environment at a time.
 *
 * Parity pins (tests/test_oracle_pins.py): every function here is checked
 * against closed forms, hand-computed poses, published known-answer vectors
 * or brute force on tiny inputs.  The neural-SDF MLP is pinned by central
 * finite differences and a one-layer closed-form gradient.
 */
#ifndef GX_ORACLE_H
#define GX_ORACLE_H
#include <stdint.h>

#define ORC_MAX_OBJ 256
#define ORC_MAX_SPHERES 32
#define ORC_BAND 1e-4 /* m: decisions this close to their threshold are "near band" */

typedef struct {
  const float* link_offset;   /* [8][3]: o_1..o_7, tool tip                 */
  const int32_t* link_axis;   /* [7]: 0 x, 1 y, 2 z                          */
  const float* q_min;         /* [7]                                         */
  const float* q_max;         /* [7]                                         */
  const float* q_rest;        /* [7]                                         */
  float dq_max, base_step, base_turn;
  int32_t n_spheres;
  const int32_t* sphere_link; /* [S]                                         */
  const float* sphere_pos;    /* [S][3] in the link frame                    */
  const float* sphere_radius; /* [S]                                         */
  const float* cam_pos;       /* [3] in the base frame                       */
  float cam_pitch, cam_near, grasp_radius, rest_clearance;
} orc_robot;

typedef struct {
  int32_t n_boxes;   const float* boxes;     /* [B][6] min xyz, max xyz     */
  int32_t n_verts;   const float* verts;     /* [V][3]                      */
  int32_t n_tris;    const int32_t* tris;    /* [T][3]                      */
  const uint32_t* tri_rgb;                   /* [T]                         */
  int32_t n_supports; const float* supports; /* [P][5] x0 z0 x1 z1 top      */
  float grid_origin[3]; float grid_h; int32_t grid_dims[3];
  float spawn[4];                            /* x0 z0 x1 z1                 */
} orc_scene;

typedef struct {
  int32_t n_verts; const float* verts;       /* unit instance mesh          */
  int32_t n_tris;  const int32_t* tris;
  const uint32_t* obj_rgb;                   /* [ORC_MAX_OBJ] colours       */
  const uint32_t* robot_rgb;                 /* [ORC_MAX_SPHERES] colours of the
                                                robot's spheres; NULL: the
                                                robot body is not rendered   */
} orc_objmesh;

typedef struct {
  double base[3];           /* x, z, yaw                                    */
  double q[7];
  int32_t held;             /* -1: nothing held                             */
  double c_off[3];          /* held object centre in the tool-tip frame     */
  double p_pre[3];          /* held object's resting position before grasp  */
  int32_t n_obj;
  double obj[ORC_MAX_OBJ][4]; /* x y z rho                                  */
  int32_t step_count;
  int32_t episode;
  /* rearrangement task (object 0 is the target) */
  double goal[3];           /* goal position of the target                  */
  double obj_start[3];      /* the target's position at the episode start   */
  double prev_a[7];         /* previous step's joint actions (clipped)      */
  double prev_d, prev_e;    /* previous tip-target, target-goal distances   */
  /* object model (appendix "Additional Collision-Detection Details"): 0 =
   * objects are spheres of radius obj[j][3]; 1 = resting objects are boxes
   * standing upright (half extents box[j][0..2], yaw box[j][3]; obj[j][3]
   * is then the bounding radius |h|) and a grasped box is carried as a set
   * of eight spheres, turning with the tool (r_off: its rotation in the
   * tool frame, row-major). */
  int32_t boxes;
  double box[ORC_MAX_OBJ][4];
  double r_off[9];
} orc_state;

typedef struct {
  uint32_t contact_mask;    /* bit i robot sphere i, bit 30 attached object */
  uint8_t flags;            /* 1 static, 2 object, 4 attached               */
  uint8_t event;            /* 0 none 1 grasp 2 miss 3 landed 4 restored    */
  uint8_t reverted;
  uint8_t pad;
  int32_t near_band;        /* decisions within ORC_BAND of threshold       */
  double ee[3];
  double cam_R[9];          /* camera-to-world, columns right, up, forward  */
  double cam_t[3];
  double reward;            /* App. "Additional Task Details", r_t          */
  double task_obs[12];      /* base frame: start - base, goal - base,
                               start - tip, goal - tip                      */
  uint8_t success;
  uint8_t pad2[7];
} orc_step_out;

typedef struct {
  int32_t near_band;
  int32_t failed;           /* placements that used all tries               */
} orc_reset_out;

typedef struct {
  int64_t tris_setup;       /* front-facing triangles reaching the image    */
  int64_t frags_covered;    /* pixel centres strictly inside them           */
  int64_t ambiguous;
  int64_t overflow;
} orc_render_stats;

#ifdef __cplusplus
extern "C" {
#endif
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_box_sdf(const double p[3], const float box[6]);
double orc_grid_node(const orc_scene* s, int i, int j, int k);
int orc_grid_query(const orc_scene* s, const double c[3], double* d, double* edge);
void orc_fk(const orc_robot* rb, const double base[3], const double q[7],
            double links[8][12], double ee[12], double cam[12]);
void orc_sphere_centres(const orc_robot* rb, const double base[3], const double q[7],
                        double out[][3]);
void orc_step(const orc_robot* rb, const orc_scene* sc, orc_state* st, const float act[11],
              orc_step_out* out);
/* Options of the general step.  dhat != NULL: the neural-SDF static test
 * (see orc_step_nsdf); slide: the sliding heuristic (contact_flags bit 8 when
 * it moved the base); place_jitter: the object placing heuristic on release
 * (event 5 when a jittered landing was found), drawing from Philox with key
 * `seed` and counter (env, step, k, 0x4A495454). */
typedef struct {
  const double* dhat;
  double margin, band;
  int32_t slide, place_jitter;
  uint64_t seed;
  int32_t env;
  int32_t column;          /* 1: static test on the column grid             */
} orc_step_opts;
/* Column grid (see gx_oracle.c): working-set radius index for r, columns
 * per axis, free spans of column (i, k) at radius index ri, and the sphere
 * test. */
int orc_column_radius_index(double r);
void orc_column_dims(const orc_scene* s, int32_t dims[2]);
int orc_column_spans(const orc_scene* s, int ri, int i, int k, double spans[][2], int cap);
int orc_column_contact(const orc_scene* s, const double c[3], double r, int* nb);
void orc_step_ex(const orc_robot* rb, const orc_scene* sc, orc_state* st, const float act[11],
                 const orc_step_opts* opt, orc_step_out* out);
int orc_grid_gradient(const orc_scene* s, const double c[3], double g[3]);
/* The step with the neural-SDF static test: dhat[i] is the predicted
 * distance at candidate sphere i (i < n_spheres; 30 = held object).  Outside
 * the lattice box is contact; dhat - r >= margin is free; else the grid
 * decides.  Predictions within `band` of the margin count as near band. */
void orc_step_nsdf(const orc_robot* rb, const orc_scene* sc, orc_state* st, const float act[11],
                   const double* dhat, double margin, double band, orc_step_out* out);
/* Candidate sphere centres and radii of the step that `act` proposes (robot
 * spheres 0..n_spheres-1, held object at 30); active[i] marks the used ones. */
void orc_candidate_spheres(const orc_robot* rb, const orc_state* st, const float act[11],
                           double c[31][3], double r[31], int32_t active[31]);
void orc_reset(const orc_robot* rb, const orc_scene* sc, orc_state* st, uint64_t seed,
               int32_t env, int32_t n_obj, float rho_min, float rho_max, orc_reset_out* out);
/* Oriented boxes (st->boxes = 1): the exact distance from c to box j
 * (negative inside), the box-frame coordinates of c, the eight carried
 * spheres of a box (centres in its frame, common radius min(h)), and the
 * overlap of two upright boxes (separating axes in the ground plane plus
 * the vertical intervals; strict). */
double orc_box_distance(const orc_state* st, int j, const double c[3]);
void orc_box_local(const double p[3], double yaw, const double c[3], double q[3]);
double orc_box_spheres(const double h[3], double centres[8][3]);
int orc_boxes_overlap(const double pa[3], const double ba[4], const double pb[3],
                      const double bb[4], int* nb);
double orc_snap(const orc_scene* s, const double p[3], double target, int* ok, int* near_band);
void orc_render(const orc_robot* rb, const orc_scene* sc, const orc_objmesh* om,
                const orc_state* st, int32_t W, int32_t H, double eps_px, double tol_rel,
                double cos_min, double* depth, uint32_t* rgb, uint8_t* ambiguous,
                int32_t* winner, orc_render_stats* stats);
/* orc_render that also reports, per pixel, |cos| between the view ray and
 * the winning surface's normal (1 where nothing is hit). */
void orc_render_cos(const orc_robot* rb, const orc_scene* sc, const orc_objmesh* om,
                    const orc_state* st, int32_t W, int32_t H, double eps_px, double tol_rel,
                    double cos_min, double* depth, uint32_t* rgb, uint8_t* ambiguous,
                    int32_t* winner, orc_render_stats* stats, double* cos_out);

/* Neural-SDF training sample i: even i uniform over the lattice box, odd i
 * the first of at most 64 uniform draws with |d| < band; label = grid d.
 * Returns the draw index used. */
int orc_nsdf_sample(const orc_scene* s, uint64_t seed, uint32_t scene, uint32_t i, double band,
                    double p[3], double* d, int* near_band);

/* Neural SDF (Fourier-feature MLP) in FP64: forward and backward.  With
 * orc_mlp_set_bf16_operands(1) every value fed to a BF16 matrix product
 * (features, hidden activations, hidden-layer gradients) is rounded to the
 * nearest BF16 first, as the tensor-core kernels do; sums stay FP64. */
void orc_mlp_set_bf16_operands(int on);
double orc_mlp_forward(const double* B /*[F][3]*/, int F, const double* const* W,
                       const double* const* b, const int* dims, int n_layers, const double x[3],
                       double* acts /* optional scratch: sum(dims) */);
double orc_mlp_loss_grad(const double* B, int F, const double* const* W, const double* const* b,
                         const int* dims, int n_layers, const double* X /*[n][3]*/,
                         const double* y /*[n]*/, int n, double clamp_lo, double clamp_hi,
                         double* const* gW, double* const* gb);
/* First-order bound of |BF16-operand kernel - plain FP64 network| at x (the
 * operands rounded to BF16, FP32 sums, features within feat_err); returns
 * the plain network's d(x) and the bound's operand, feature and FP32 parts
 * in terms[0..2] (terms[3]: the operand part's standard deviation for
 * independent uniform roundings, a typical size rather than a bound). */
double orc_mlp_rounding_bound(const double* B, int F, const double* const* W,
                              const double* const* b, const int* dims, int n_layers,
                              const double x[3], double feat_err, double terms[4]);
#ifdef __cplusplus
}
#endif
#endif
