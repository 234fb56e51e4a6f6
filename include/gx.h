/*
 * gx.h -- C ABI of the batched environment step of Galactic
 * (arXiv 2306.07552) on one B300 GPU.
 *
 * One call advances every environment by one step (Sec. 3.1 "Batching": one
 * simulator instance steps all environments and shares scene assets across
 * them).  A step applies the action offsets to the robot state, runs forward
 * kinematics, tests the robot's collision spheres against the static scene
 * and the movable objects, rejects all robot motion on contact, grasps or
 * releases objects (Sec. 3.2 "Approximate Kinematic Simulation"), and renders
 * each environment's egocentric depth and RGB camera (Sec. 3.1; 128x128,
 * 90-degree FOV, Sec. 4.1) into caller-owned device buffers, which is the
 * zero-copy hand-off of Sec. 3.1.
 *
 * Conventions (all sides):
 *   - world is Y-up, the floor is the XZ plane, units are metres and radians;
 *   - robot base frame: Trans(x, 0, z) Ry(yaw); "forward" is +x of that frame;
 *   - camera space: x right, y up, z forward; pixel (i, j) has its centre at
 *     (i + 0.5, j + 0.5), i to the right, j downward; focal length W/2
 *     (90-degree horizontal FOV); depth is planar camera-space z, 0 = no hit;
 *   - images are row-major [env][row][col] (RGB: [env][row][col][3], R first).
 *
 * Errors: every entry point returns a gx_status.  Arguments the host can
 * check are validated before any GPU work and return GX_EINVAL with nothing
 * launched.  Problems only the device can see (non-finite actions, which are
 * then treated as 0; placements that used all their tries) set a device error
 * word; it is read without blocking on the next gx_step/gx_reset and reported
 * as GX_EDEVICE there or by gx_sync.  The library never traps the GPU and
 * every device loop is bounded.  gx_last_error() gives a message.
 *
 * Threading: one context per host thread.  Calls are asynchronous on the
 * caller's stream (a cudaStream_t passed as void*; NULL = legacy default
 * stream).  Scene sets are immutable after creation and may be shared by
 * several contexts; a scene set must outlive the contexts using it.
 */
#ifndef GX_H
#define GX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GX_OK = 0,
  GX_EINVAL = 1,   /* bad argument, detected on the host; nothing launched   */
  GX_ENOMEM = 2,   /* device or host allocation failed                        */
  GX_ECUDA = 3,    /* a CUDA runtime call failed                              */
  GX_EDEVICE = 4,  /* the device error word was set (see gx_last_error)       */
  GX_ESTATE = 5    /* call not valid in the current state                     */
} gx_status;

/* device error word bits (gx_device_error) */
#define GX_DEV_NONFINITE_ACTION 0x1u  /* some action was NaN/Inf; used 0     */
#define GX_DEV_PLACEMENT_FAILED 0x2u  /* a reset placement used all 64 tries
                                         and kept the last one; reported by
                                         gx_device_error only (no GX_EDEVICE) */

#define GX_MAX_OBJECTS 256
#define GX_MAX_SPHERES 31

/* Robot description (FP32, host memory, copied at gx_create).
 * Sec. 3.2: the robot is an articulated chain moved kinematically; each link
 * is approximated by hand-placed spheres (appendix "Additional
 * Collision-Detection Details").  Link k's frame sits at joint k:
 *   T_0 = Trans(x, 0, z) Ry(yaw),  T_k = T_{k-1} Trans(o_k) Rot(axis_k, q_k),
 *   tool tip T_ee = T_7 Trans(o_tip),  camera T_cam = T_0 Trans(cam_pos) M,
 * M having columns right (0,0,-1), up (-sin p, cos p, 0), forward
 * (cos p, sin p, 0) for pitch p. */
typedef struct {
  float link_offset[8][3];  /* o_1..o_7, then o_tip                         */
  int32_t link_axis[7];     /* 0 = x, 1 = y, 2 = z                           */
  float q_min[7], q_max[7]; /* joint limits (rad)                            */
  float q_rest[7];          /* joints after a reset                          */
  float dq_max;             /* joint offset per step at |action| = 1 (rad)   */
  float base_step;          /* base translation at |action| = 1 (App. A: 0.10 m) */
  float base_turn;          /* base rotation at |action| = 1 (App. A: 5 deg) */
  int32_t n_spheres;        /* <= 30: bit 30 of contact masks is reserved    */
  int32_t sphere_link[GX_MAX_SPHERES];   /* 0 = base, k = link k            */
  float sphere_pos[GX_MAX_SPHERES][3];   /* centre in the link frame        */
  float sphere_radius[GX_MAX_SPHERES];
  float cam_pos[3];         /* head camera in the base frame                 */
  float cam_pitch;          /* rad; negative looks down                      */
  float cam_near;           /* near plane (m), > 0                           */
  float grasp_radius;       /* suction sphere at the tool tip (Sec. 3.2: 0.03 m) */
  float rest_clearance;     /* resting objects sit this far above contact (m) */
} gx_robot;

/* One static scene, host memory, read during gx_scene_set_create only.
 * boxes: the solids the signed-distance grid is built from (union of boxes);
 * verts/tris/tri_rgb: the triangles rendered (front face counter-clockwise
 * seen from outside, so outward normal = (v1-v0) x (v2-v0));
 * supports: rectangles objects are placed on at reset (x0 z0 x1 z1 top_y);
 * grid: node (i,j,k) at origin + (i,j,k) * h, dims = (nx, ny, nz);
 * spawn: x0 z0 x1 z1 region sampled for the robot base at reset. */
typedef struct {
  int32_t n_boxes;    const float* boxes;     /* [n_boxes][6] min xyz max xyz */
  int32_t n_verts;    const float* verts;     /* [n_verts][3]                 */
  int32_t n_tris;     const int32_t* tris;    /* [n_tris][3]                  */
  const uint32_t* tri_rgb;                    /* [n_tris] 0x00RRGGBB          */
  int32_t n_supports; const float* supports;  /* [n_supports][5], >= 1        */
  float grid_origin[3];
  float grid_h;                               /* node spacing (m)             */
  int32_t grid_dims[3];                       /* each >= 2                    */
  float spawn[4];
} gx_scene_desc;

/* Instance mesh for free objects (unit circumradius; scaled by each object's
 * radius) and one colour per object index; robot_rgb colours the robot's
 * collision spheres when a context renders the robot body (the same mesh,
 * instance slots GX_MAX_OBJECTS + sphere index). */
typedef struct {
  int32_t n_verts;    const float* verts;     /* [n_verts][3], <= 32          */
  int32_t n_tris;     const int32_t* tris;    /* [n_tris][3], <= 32           */
  uint32_t obj_rgb[GX_MAX_OBJECTS];
  uint32_t robot_rgb[32];
} gx_object_mesh;

typedef struct gx_scene_set gx_scene_set;
typedef struct gx_ctx gx_ctx;

typedef struct {
  int32_t n_envs;          /* >= 1                                            */
  int32_t img_w, img_h;    /* multiples of 32, <= 256                         */
  int32_t depth_fp16;      /* 0: depth as float32, 1: as IEEE half            */
  int32_t render_rgb;      /* 0: skip the RGB image                           */
  int32_t n_objects;       /* free objects per environment, <= 256            */
  float obj_radius_min, obj_radius_max;   /* object radius drawn at reset     */
  uint64_t seed;           /* Philox key for resets                           */
  const int32_t* env_scene; /* host [n_envs] scene per env; NULL: env i uses
                               scene floor(i * n_scenes / n_envs)             */
  int32_t small_tri_px;    /* triangles whose clipped bounding box exceeds this
                              many pixels are scanned block-wise by a warp
                              instead of by fragment expansion (0: only those
                              128 px or larger, and near-clipped ones)        */
  int32_t use_graph;       /* 1: replay the step as a captured CUDA graph     */
  int32_t profile;         /* bit 0: time each kernel with CUDA events on the
                              caller's stream (disables graph replay);
                              bit 1: also count rasteriser work (slower);
                              bit 2: count neural-SDF decisions against the
                              grid-only rule (evaluates both; slower);
                              bit 3: NVTX ranges around gx_reset, gx_step,
                              gx_step_reset and each kernel's enqueue (for
                              timelines and ncu --nvtx filters);
                              bit 4: count step events (gx_step_counters;
                              not with object_boxes)                          */
  int32_t sdf_mode;        /* 0: static test on the distance grid;
                              2: on the column grid (appendix "Additional
                              Collision-Detection Details"): per working-set
                              radius {1.5, 5, 12} cm, columns 3 cm apart in XZ
                              over the grid box holding the free spans of a
                              sphere centre's height; a sphere uses the
                              smallest working radius R not below its own r at
                              the nearest column, the spans widened by R - r
                              at both ends (release, reset and the sliding
                              heuristic keep the distance grid);
                              1: neural SDF (every scene an environment uses
                              needs weights, gx_nsdf_set_weights): the grid is
                              consulted only where the predicted clearance
                              d - r is below sdf_margin, or not finite; a
                              centre outside the grid box is contact          */
  float sdf_margin;        /* metres, >= 0 (e.g. 0.02)                        */
  int32_t broadphase;      /* 1: robot spheres meet only the objects listed in
                              one cell of four offset regular grids per env
                              (appendix "Additional Collision-Detection
                              Details"; cells 0.5 m, 12 objects each, fuller
                              cells brute force); results are unchanged       */
  int32_t render_robot;    /* 1: the robot's collision spheres are rendered
                              (instanced like the objects, robot_rgb)        */
  int32_t heuristics;      /* the paper's heuristics (appendix "Description of
                              Heuristics"), bit 0: sliding -- a colliding
                              candidate base is jittered in the ground plane
                              at most 3 times, along the penetration-weighted
                              outward normals by the deepest penetration + 1 mm
                              (contact_flags bit 3 = 8 when it moved); bit 1:
                              object placing -- a failed release is jittered
                              at most 6 times by 2 rho away from overlapped
                              objects (random turn in [-pi/4, pi/4), Philox on
                              env, step, k, 0x4A495454 with the reset seed) and
                              re-cast down (event 5 when that lands)          */
  int32_t raster_order;    /* rasteriser work order: 0 chosen at creation
                              (costliest scene first when the scenes' cluster
                              counts differ by more than 1.5x, else index
                              order), 1 index order, 2 costliest scene first;
                              gx_autotune may change it                       */
  int32_t env_offset;      /* global index of this context's environment 0:
                              the Philox counters of resets and placing jitters
                              use env_offset + local index, so a batch split
                              over several contexts (one per GPU) draws exactly
                              what one context over the whole batch draws    */
  int32_t object_boxes;    /* the paper's object model (appendix "Additional
                              Collision-Detection Details"): 0 objects are
                              spheres; 1 resting objects are upright oriented
                              boxes (half extents drawn in [obj_radius_min,
                              obj_radius_max) per axis, yaw uniform; robot
                              spheres tested by the exact sphere-box distance
                              in the box frame) and a grasped box is carried
                              as eight spheres of radius min(h) at its inset
                              corners, turning with the tool; release stands
                              it upright about its heading and rests it on the
                              highest landing of its four bottom spheres unless
                              it would overlap another box (separating axes),
                              else restores it.  Boxes render as cubes mapped
                              by rotation x half extents.  Only with sdf_mode 0
                              and without heuristics, broad-phase or robot-body
                              rendering (GX_EINVAL otherwise)                 */
  int32_t raster_warps;    /* warps per rasteriser CTA: 8 (three CTAs per SM),
                              12 (two per SM; not with object_boxes), 6 (four
                              per SM; not with fused_step, object_boxes or
                              occlusion_cull), 7 (four per SM; not with
                              fused_step or occlusion_cull); 0: 7 where
                              offered, else 8; gx_autotune may change it      */
  int32_t occlusion_cull;  /* 1: the rasteriser culls clusters by occlusion in
                              two phases per environment: first the clusters
                              it showed in its previous image (one bit per
                              cluster, kept by the context), then the others
                              and the objects only where the depth bound of
                              some 8x8 tile they touch (the farthest of that
                              tile's pixels so far) could still let them win;
                              the bits are rewritten from the final image.
                              Images are identical to the unculled ones; with
                              it, gx_autotune also times the setting without
                              it.  8 warps per CTA; not with fused_step or
                              object_boxes (GX_EINVAL)                        */
  int32_t fused_step;      /* 1: each step (gx_step, gx_step_reset) is one
                              cooperative persistent launch of the
                              rasteriser's grid: masked resets, then physics
                              (a warp per environment), then rendering,
                              separated by grid-wide barriers with bounded
                              waits (a wait that gives up sets the device error
                              word).  Not with sdf_mode 1 or object_boxes
                              (GX_EINVAL); gx_phase_times then reports the
                              whole launch as ms[1].                          */
  int32_t static_store;    /* where the distance grid's node values come from
                              for every static test of this context (the step,
                              the neural SDF's fallback, release, reset, the
                              sliding heuristic): 0 the dense FP32 grid built
                              with the scene set; 1 the box store -- each node
                              recomputed in FP32 from the scene's solid boxes
                              as the minimum over a short per-cell list of
                              candidate boxes (cells of 16 node intervals per
                              axis, chosen so the list holds the nearest box of
                              every node of the cell), within 1e-5 m of the
                              FP64 node value for coordinates up to 20 m;
                              about 0.1% of the dense grid's bytes, so a scene
                              set created without dense grids
                              (gx_scene_set_create_ex) can serve it; not with
                              fused_step (GX_EINVAL)                          */
} gx_config;

/* Outputs of one step, device memory owned by the caller (e.g. torch
 * tensors), written in place.  NULL members are skipped, except that depth
 * is required.  pose: [n][16] = q0..q6, holding (0/1), base x, base z, yaw,
 * tool tip x, y, z (world), step counter, 0. */
typedef struct {
  void* depth;             /* [n][h][w] float32 or half                       */
  uint8_t* rgb;            /* [n][h][w][3] (only if render_rgb)               */
  float* pose;             /* [n][16]                                         */
  float* obj_pos;          /* [n][n_objects][4] x y z radius                  */
  int32_t* held;           /* [n] held object index or -1                     */
  uint32_t* contact_mask;  /* [n] bit i robot sphere i, bit 30 held object    */
  uint8_t* contact_flags;  /* [n] 1 static, 2 object, 4 held object           */
  uint8_t* event;          /* [n] 0 none, 1 grasped, 2 grasp missed,
                              3 released and landed, 4 released and restored,
                              5 released and landed after placing jitters    */
  /* rearrangement task (object 0 is the target; its goal is drawn at reset
   * on a support top): */
  float* reward;           /* [n] 10 success + 5 pick + (d_{t-1} - d_t)
                              + (e_{t-1} - e_t) - 0.001 sum_k (a_k - a'_k)^2,
                              d tip-target, e target-goal distance, a / a' this
                              and the previous step's clipped joint actions;
                              success: stop >= 0.5 with the target released
                              within 0.15 m of the goal; pick: the target was
                              just grasped (App. "Additional Task Details")  */
  float* task_obs;         /* [n][12] in the base frame: target start - base,
                              goal - base, target start - tip, goal - tip      */
  uint8_t* success;        /* [n]                                              */
} gx_outputs;

/* Builds the device copies of `n_scenes` scenes: the FP32 signed-distance
 * grid of each (computed on the GPU in FP64 from the boxes, then rounded),
 * the triangle clusters used by the rasteriser, supports and spawn regions,
 * and the object instance mesh.  Blocks until done.
 * Errors: GX_EINVAL (NULL pointers, counts out of range), GX_ENOMEM, GX_ECUDA. */
gx_status gx_scene_set_create(const gx_scene_desc* scenes, int32_t n_scenes,
                              const gx_object_mesh* mesh, gx_scene_set** out);
gx_status gx_scene_set_destroy(gx_scene_set* set);

/* Which static structures gx_scene_set_create_ex builds (gx_scene_set_create
 * builds all); the paper builds its static collision structure offline from
 * the scene (appendix "Additional Collision-Detection Details").  The box store (gx_config.static_store 1) is always built; it
 * is the distance grid's definition evaluated on demand, so a set without
 * dense grids keeps every static test of the step, and a set without column
 * grids only loses sdf_mode 2.  Training samples (gx_nsdf_samples,
 * gx_nsdf_train) read the dense grid when the set has it, else the box
 * store. */
typedef struct {
  int32_t dense_grid;      /* 1: the dense FP32 grid [nz][ny][nx] per scene   */
  int32_t column_grid;     /* 1: the column grid per scene (sdf_mode 2)       */
} gx_scene_options;
/* Errors as gx_scene_set_create; GX_EINVAL for options other than 0 or 1. */
gx_status gx_scene_set_create_ex(const gx_scene_desc* scenes, int32_t n_scenes,
                                 const gx_object_mesh* mesh, const gx_scene_options* options,
                                 gx_scene_set** out);

/* (No counterpart in the paper: memory accounting.)  Device bytes of one
 * scene's structures, written to the host array bytes: bytes[0] dense distance grid (0
 * when not built), [1] box store (boxes and candidate lists), [2] column grid
 * (0 when not built), [3] render clusters (headers, vertices, triangles,
 * colours), [4] neural-SDF weights (0 before gx_nsdf_set_weights), [5]
 * neural-SDF FP32 master copy kept for training (0 when none). */
gx_status gx_scene_bytes(const gx_scene_set* set, int32_t scene, uint64_t bytes[6]);

/* (No counterpart in the paper: inspection of the box store.)
 * The box store's candidate lists of one scene (gx_config.static_store 1),
 * built on the host exactly as gx_scene_set_create builds them; no device is
 * touched.  The lattice's node intervals are grouped 16 per axis into cells,
 * dims[0..2] of them along x, y, z; cell (cx, cy, cz) has index
 * (cz * dims[1] + cy) * dims[0] + cx and lists, as box indices
 * ids[offsets[c] .. offsets[c + 1]), every box that can be the nearest one
 * at some node of the cell (nodes 16c .. 16c + 16 per axis).  Call once with
 * offsets and ids NULL for dims and *n_ids, then with offsets [cells + 1] and
 * ids [*n_ids] (host buffers).  GX_EINVAL for a scene without boxes or with a
 * bad lattice. */
gx_status gx_box_store_lists(const gx_scene_desc* scene, int32_t dims[3], uint32_t* offsets,
                             uint16_t* ids, uint64_t* n_ids);

/* The static scene's distance query of the step (appendix "Additional
 * Collision-Detection Details"; the grid's trilinear value) on its own.
 * Static distance at n points (device pts [n][3]) into dist (device [n]):
 * the trilinear interpolation of the scene's distance grid whose nodes come
 * from `store` (0 dense grid, 1 box store; see gx_config.static_store); NaN
 * where a point lies outside the lattice box (contact for the step).
 * Asynchronous on `stream`.  GX_EINVAL for store 0 on a set without dense
 * grids. */
gx_status gx_static_distance(const gx_scene_set* set, int32_t scene, int32_t store,
                             const float* pts, int32_t n, float* dist, void* stream);

/* Allocates the structure-of-arrays state for cfg->n_envs environments on
 * the current device, borrowing `set`.  All environments start unplaced:
 * call gx_reset (mask NULL) before the first gx_step.
 * Errors: GX_EINVAL, GX_ENOMEM, GX_ECUDA. */
gx_status gx_create(const gx_scene_set* set, const gx_robot* robot, const gx_config* cfg,
                    gx_ctx** out);
void gx_destroy(gx_ctx* ctx);

/* Starts a new episode in every environment whose byte in env_mask (device,
 * [n_envs]) is non-zero, or in all when env_mask is NULL: objects are placed
 * on support tops and the robot base in free space by rejection sampling
 * (at most 64 Philox4x32-10 draws each, keyed by (seed, env, episode)), the
 * joints go to q_rest and nothing is held.  Asynchronous. */
gx_status gx_reset(gx_ctx* ctx, const uint8_t* env_mask, void* stream);

/* Advances every environment by one step.  actions: device [n_envs][11]
 * float32 = base forward, base turn (+1 clockwise seen from above), 7 joint
 * offsets, grasp (>= 0.5 grasps, else releases), stop (ignored); each value
 * is clipped to [-1, 1] (App. A).  Asynchronous on `stream`. */
gx_status gx_step(gx_ctx* ctx, const float* actions, const gx_outputs* out, void* stream);

/* gx_reset(env_mask) followed by gx_step(actions) in one call: the
 * environments whose byte in env_mask (device, [n_envs]; NULL: none) is
 * non-zero start a new episode, then every environment advances one step.
 * With fused_step this is a single kernel launch; otherwise the launches of
 * the two calls.  With use_graph the whole call is replayed as one captured
 * graph (keyed on the mask, action and output pointers). */
gx_status gx_step_reset(gx_ctx* ctx, const uint8_t* env_mask, const float* actions,
                        const gx_outputs* out, void* stream);

/* Same step with HOST actions: copies the actions (pinned host memory is
 * fastest) to the device, steps into the context's own device output
 * buffers, and copies back every non-NULL member of `host_out` (host
 * buffers, same layouts as gx_outputs; depth may be NULL too).  The outputs
 * not copied stay on the device, where gx_device_outputs finds them (the
 * paper's zero-copy hand-off of observations to a policy on the GPU).
 * Blocks until the copies are complete. */
gx_status gx_step_host(gx_ctx* ctx, const float* actions_host, const gx_outputs* host_out,
                       void* stream);

/* Device pointers of the context's own output buffers that gx_step_host
 * writes (all members set once gx_step_host has run; GX_ESTATE before). */
gx_status gx_device_outputs(gx_ctx* ctx, gx_outputs* out);

/* Waits for all work of ctx and reports the device error word. */
gx_status gx_sync(gx_ctx* ctx);
uint32_t gx_device_error(gx_ctx* ctx); /* waits, returns and clears the word */

/* Environment state as one host blob (layout: see gx_state_layout). */
size_t gx_state_bytes(const gx_ctx* ctx);
gx_status gx_save_state(gx_ctx* ctx, void* host, size_t bytes);
gx_status gx_load_state(gx_ctx* ctx, const void* host, size_t bytes);
/* Byte offsets of the state arrays, in this order: base_x, base_z, yaw
 * [n] f32; q [7][n] f32; held [n] i32; c_off [3][n] f32 (held object in the
 * tool-tip frame); p_pre [3][n] f32 (its pre-grasp position); obj
 * [n][n_objects][4] f32 (x, y, z, radius; for box objects the bounding
 * radius); step [n] i32; episode [n] i32; task [n][16] f32 (goal xyz,
 * target start xyz, previous joint actions [7], previous tip-target and
 * target-goal distances, unused); box [n][n_objects][4] f32 (box objects:
 * half extents xyz and resting yaw; unused with spheres); r_off [9][n] f32
 * (box objects: the held box's rotation in the tool frame, row-major).
 * Each array starts on a 256-byte boundary of the blob. */
#define GX_STATE_ARRAYS 13
gx_status gx_state_layout(const gx_ctx* ctx, size_t offsets[GX_STATE_ARRAYS]);

/* Per-kernel device time recorded since the previous call when the context
 * was created with profile bit 0 set: ms[0] physics (both passes when
 * sdf_mode is 1), ms[1] rasteriser, ms[2] reset, ms[3] neural-SDF queries;
 * launches[k] the number of timed launches.  Waits for the device. */
gx_status gx_phase_times(gx_ctx* ctx, double ms[4], int64_t launches[4]);

/* Rasteriser work counters accumulated since the previous call (contexts
 * created with profile bit 1), then cleared: clusters tested, clusters drawn,
 * triangles seen, front-facing, rasterised by fragment expansion, pixels
 * they expand to, rasterised per warp, 8x4 blocks the warps scanned,
 * near-clipped, fragments written, mbarrier polls, expansion passes,
 * 32-triangle set-up rounds, expansion slots (runs of up to four pixels),
 * clusters skipped by the occlusion test.
 * Fills out[0..n-1]; waits for the device.
 * GX_ESTATE when the context does not count. */
gx_status gx_raster_counters(gx_ctx* ctx, int64_t* out, int32_t n);

/* (No counterpart in the paper: profiling of the step of Sec. 3.2.)
 * Step event counters accumulated since the previous call (contexts created
 * with profile bit 4), then cleared: env-steps with a contact (contact mask
 * non-zero), grasps, missed grasps, releases that landed (also after placing
 * jitters), releases restored, static tests and object-pair tests within
 * 1e-4 m of their threshold (the near band of the parity tests; the static
 * ones on the distance grid or box store, whatever the context decides with),
 * sliding moves.  Fills out[0..n-1]; waits for the device.  GX_ESTATE when
 * the context does not count. */
gx_status gx_step_counters(gx_ctx* ctx, int64_t* out, int32_t n);

/* Rasteriser settings chosen by gx_autotune. */
typedef struct {
  int32_t small_tri_px;           /* as gx_config.small_tri_px (0: default)      */
  int32_t order_costliest_first;  /* 1: environments of the scenes with the most
                                     triangle clusters are rendered first       */
  int32_t raster_ctas;            /* persistent CTAs launched                    */
  float ms_per_step;              /* measured step time with these settings      */
  int32_t raster_warps;           /* warps per rasteriser CTA (6, 7, 8 or 12)    */
  int32_t occlusion_cull;         /* 1: clusters culled by occlusion             */
} gx_tune_result;

/* Times the step on this context's own state under each candidate rasteriser
 * setting -- expansion limit small_tri_px in {0, 256, 96, 48}, work order
 * {index, costliest scene first}, CTA shape {8 warps at the occupancy (three
 * CTAs per SM), 8 warps one CTA per SM fewer, 12 warps at its occupancy (two
 * per SM), 6 and 7 warps at their occupancy (four per SM; not offered with
 * occlusion culling); the fused step keeps 8 warps, box objects take 8 or 7} -- for `steps` steps each (plus one
 * warm-up), restoring the
 * state after every candidate, and keeps the fastest (written to *best when
 * not NULL).  The outputs are overwritten; the state is left as before the
 * call.  actions: device [n][11], reused for every step.  Allocates one copy
 * of the state; waits for the stream.  The context starts with the index
 * order, or the costliest-first order when its scenes' cluster counts differ
 * by more than 1.5x. */
gx_status gx_autotune(gx_ctx* ctx, const float* actions, const gx_outputs* out, int32_t steps,
                      gx_tune_result* best, void* stream);

/* (No counterpart in the paper: the autotuner is this library's.)
 * Applies a rasteriser setting found earlier by gx_autotune (for example one
 * kept in a cache keyed by the configuration and the GPU) without timing
 * anything: small_tri_px, order_costliest_first, raster_warps, raster_ctas
 * and occlusion_cull are used, ms_per_step is ignored.  Images do not depend
 * on the setting.  GX_EINVAL when the setting does not fit this context (a
 * CTA shape it cannot use, more CTAs than that shape keeps resident, occlusion
 * culling without the context's visibility bits).  Touches no device memory;
 * a captured step graph is rebuilt at the next replay. */
gx_status gx_apply_tune(gx_ctx* ctx, const gx_tune_result* setting);

/* Neural-SDF decision counters accumulated since the previous call (profile
 * bit 2):
 * out[0] static tests made, out[1] of which the grid decided, out[2]
 * decisions that differ from the grid-only rule, out[3] env-steps whose
 * contact mask differs from it.  Waits for the device.  GX_ESTATE when the
 * context does not count. */
gx_status gx_nsdf_counters(gx_ctx* ctx, int64_t out[4]);

/* The network's predictions d^ that the last step's static test used
 * (sdf_mode 1), copied into the host buffer `host` of n_values = n_envs * 32
 * floats: [env][slot], slot s < 30 robot sphere s at the candidate pose,
 * slot 30 the held object; a slot is meaningful only where that sphere was
 * tested (slot 31 and spheres without a held object are not).  NaN before
 * the first step.  Waits for the device.  GX_ESTATE when sdf_mode is not 1,
 * GX_EINVAL on a size mismatch. */
gx_status gx_nsdf_step_predictions(gx_ctx* ctx, float* host, size_t n_values);

/* ----------------------------------------------------------------------------
 * Neural SDF (not in the paper; the learned stand-in for the distance grid).
 * Per scene, a Fourier-feature MLP
 *   d(x) = W5 relu(W4 relu(W3 relu(W2 relu(W1 g(x) + b1) + b2) + b3) + b4) + b5,
 *   g(x) = [sin(2 pi B (x - c)), cos(2 pi B (x - c))],
 * B [32][3], c the centre of the scene's grid box, hidden width 128.  W1..W4
 * are stored and multiplied in BF16 on the tensor cores with FP32
 * accumulation; features and hidden activations are rounded to BF16 where
 * they enter a product; biases, W5 and b5 are FP32.
 * params layout (GX_NSDF_PARAMS floats): W1 [128][64], b1 [128], W2 [128][128],
 * b2, W3, b3, W4, b4, W5 [128], b5 [1] (row-major, rows = outputs).
 * Setting or training weights mutates the scene set: do it while no context
 * using the set is stepping. */
#define GX_NSDF_PARAMS 57985

/* Loads weights (host FP32; W1..W4 are rounded to BF16 for the kernels, the
 * FP32 values are kept as training's master copy) for one scene.  Allocates
 * the scene's device copies on first use. */
gx_status gx_nsdf_set_weights(gx_scene_set* set, int32_t scene, const float* fourier_B,
                              const float* params);
/* The weights as the kernels use them (BF16 values widened to FP32), the
 * Fourier matrix and the feature centre c (each output may be NULL except
 * params).  GX_ESTATE when the scene has no neural SDF. */
gx_status gx_nsdf_get_weights(const gx_scene_set* set, int32_t scene, float* fourier_B,
                              float* params, float* centre);
/* The FP32 master parameters (training's copy; equal to the values last
 * passed to gx_nsdf_set_weights until gx_nsdf_train changes them) into
 * params (host, GX_NSDF_PARAMS).  Waits for the device. */
gx_status gx_nsdf_get_master(const gx_scene_set* set, int32_t scene, float* params);
/* d(x) for n points (device [n][3] world coordinates) into dist (device [n]).
 * Asynchronous on `stream`. */
gx_status gx_nsdf_query(const gx_scene_set* set, int32_t scene, const float* pts, int32_t n,
                        float* dist, void* stream);

/* Training-sample stream of one scene (workload definition): sample i (0 <=
 * i < 2^32) is, for even i, a uniform point of the scene's grid box and, for
 * odd i, the first of at most 64 such points whose grid distance has
 * |d| < near_band (the last one when none has); point t of sample i comes from
 * Philox4x32-10 on counter (i, scene, t, 0x4E534446) with key (seed low 32
 * bits, seed high 32 bits), coordinate = origin + ((word >> 8) / 2^24) *
 * (dims - 1) * h.  Label = trilinear grid distance.  Writes samples
 * [first, first + n) to pts (device [n][3]) and dist (device [n]);
 * asynchronous on `stream`. */
gx_status gx_nsdf_samples(const gx_scene_set* set, int32_t scene, uint64_t seed, int64_t first,
                          int64_t n, float near_band, float* pts, float* dist, void* stream);

/* Gradient of the mean L1 loss (1/n) sum |d(x_i) - clamp(y_i, lo, hi)| with
 * respect to the GX_NSDF_PARAMS parameters (layout as above), evaluated with
 * the scene's current weights on n points (device pts [n][3], labels [n]),
 * into grad (device [GX_NSDF_PARAMS]) and the loss into *loss (device, may be
 * NULL).  BF16 operands as in the forward; the gradients of hidden
 * pre-activations are rounded to BF16 where they enter a product.  Allocates
 * its workspace, waits for the stream; GX_EDEVICE when a bounded wait inside
 * a kernel gave up. */
gx_status gx_nsdf_grad(gx_scene_set* set, int32_t scene, const float* pts, const float* labels,
                       int32_t n, float clamp_lo, float clamp_hi, float* grad, float* loss,
                       void* stream);

typedef struct {
  int64_t n_samples;   /* training set size (samples 0 .. n_samples-1), <= 2^32 */
  int32_t batch;       /* samples per Adam step; batch t = samples t*batch ..   */
                       /* (t+1)*batch-1, indices modulo n_samples              */
  int32_t steps;       /* Adam steps                                            */
  float lr;            /* peak rate; step t uses lr (1 + cos(pi t / steps)) / 2 */
  float beta1, beta2, eps;   /* Adam (Kingma and Ba 2015)                       */
  float clamp_lo, clamp_hi;  /* labels clamped to [lo, hi] (m)                  */
  float near_band;     /* sample stream parameter (m), as gx_nsdf_samples       */
  uint64_t seed;       /* sample stream seed                                    */
} gx_train_params;

/* Trains the scene's network from its current weights (gx_nsdf_set_weights
 * must have been called): draws the sample set, then `steps` Adam steps with
 * fresh moments.  FP32 master parameters; the BF16 copy the kernels read is
 * rewritten after every step.  loss_host (host, [steps], may be NULL)
 * receives each step's loss.  Allocates n_samples * 16 bytes plus the batch's
 * workspace (245,760 bytes per 128 samples) and frees them; waits for the
 * stream. */
gx_status gx_nsdf_train(gx_scene_set* set, int32_t scene, const gx_train_params* params,
                        float* loss_host, void* stream);

/* (Not in the paper: the learned part's training, as gx_nsdf_train.)
 * Steps first_step .. first_step + n_steps - 1 of the training run `params`
 * defines (its cosine rate over params->steps, bias corrections and batches
 * of those step numbers), from the scene's current FP32 master parameters and
 * the Adam moments in moments_in (host [2][GX_NSDF_PARAMS], first moments
 * then second; NULL: zero, as at step 0); the moments after the last step go
 * to moments_out (host, may be NULL).  A run split into consecutive ranges,
 * the moments carried from one to the next, gives the same parameters bit
 * for bit as gx_nsdf_train over the whole run, also across processes (keep
 * gx_nsdf_get_master and the moments; restore them with gx_nsdf_set_weights
 * and moments_in): training checkpoints.  loss_host: [n_steps] or NULL.
 * GX_EINVAL when the range leaves [0, params->steps); allocation and errors
 * as gx_nsdf_train. */
gx_status gx_nsdf_train_steps(gx_scene_set* set, int32_t scene, const gx_train_params* params,
                              int32_t first_step, int32_t n_steps, const float* moments_in,
                              float* moments_out, float* loss_host, void* stream);

/* Column grid of a scene (built with the scene set; see sdf_mode 2): columns
 * per axis (dims[0] along x, dims[1] along z) and its size in device bytes
 * (bytes may be NULL). */
gx_status gx_column_info(const gx_scene_set* set, int32_t scene, int32_t dims[2], uint64_t* bytes);
/* Free spans (lo, hi pairs, host float [cap][2]) of column (i, k) at
 * working-set radius index 0, 1, 2 (1.5, 5, 12 cm); returns the number of
 * spans (only the first cap are copied), -1 on a bad argument.  Waits for
 * the device. */
int32_t gx_column_spans(const gx_scene_set* set, int32_t scene, int32_t radius_index, int32_t i,
                        int32_t k, float* spans, int32_t cap);

/* Renders depth (and RGB when rgb != NULL) for n environments without
 * allocating any device memory.  The paper has no counterpart: this serves
 * callers that cannot call cudaMalloc when they need images -- code in a
 * section where device allocation is forbidden or would stall (real-time
 * loops, allocation-free serving paths, hosts that only allow allocation at
 * start-up) or embedders that have spent their memory budget.  Instead of the
 * framebuffer slots a context allocates, it uses a fixed 16 MiB scratch array
 * built into the library, which every GPU that loads the library keeps until
 * the process exits; with it at most 16 MiB / (img_w * img_h * 8) CTAs render
 * at once, so it is slower than gx_step on large batches.
 * Inputs (device memory, caller-owned): env_scene [n] scene index per env;
 * cam [n][12] camera-to-world rotation, row-major with columns right, up,
 * forward, then the eye position; obj [n][n_objects][4] object centre and
 * radius.  Outputs: depth [n][img_h][img_w] float32 (or half when depth_fp16),
 * rgb [n][img_h][img_w][3] (optional).  Image sides must be multiples of 32
 * and at most 256 (larger sizes return GX_EINVAL); n_objects <= 256.  The
 * scene set must live on the current device (else GX_EINVAL).  The images
 * are those of a gx_step with render_robot 0: scene triangles and the
 * objects given, not the robot body.
 * The first call on a device (the current one) sets the scratch up
 * synchronously; make that first call before any stream capture.  Every call
 * shares the same scratch and clears what it needs at the start, so calls
 * that overlap on the GPU (other streams, other host threads) race: order
 * them on one stream.  Asynchronous on `stream` after the first call.
 * Problems only the device sees are recorded in an error word inside the
 * scratch and accumulate over calls until gx_render_noalloc_error reads
 * them: an env_scene value outside [0, n_scenes) draws that environment
 * empty (depth 0, RGB 0) and sets GX_NOALLOC_BAD_SCENE; a bounded wait that
 * gave up leaves some images incomplete and sets GX_NOALLOC_WAIT_TIMEOUT. */
gx_status gx_render_noalloc(const gx_scene_set* set, int32_t n, const int32_t* env_scene,
                            const float* cam, const float* obj, int32_t n_objects, int32_t img_w,
                            int32_t img_h, float cam_near, void* depth, int32_t depth_fp16,
                            uint8_t* rgb, void* stream);

/* Device error bits of gx_render_noalloc calls on the current device since
 * the previous query: waits for the whole device (every stream), copies the
 * word into *bits (may be NULL), clears it, and returns GX_EDEVICE with a
 * message when any bit is set, GX_OK otherwise (also before any call).
 * Allocates nothing. */
#define GX_NOALLOC_WAIT_TIMEOUT 0x100u
#define GX_NOALLOC_BAD_SCENE 0x200u
gx_status gx_render_noalloc_error(uint32_t* bits);

/* (No counterpart in the paper: memory budgeting.)
 * Caps the device memory this library allocates -- scene sets, contexts,
 * training workspaces, on every device, for the whole process -- at `bytes`
 * (0: no cap, the default).  An allocation that would pass the cap fails as
 * an exhausted device would: the call returns GX_ENOMEM and releases what it
 * had allocated.  Memory already held keeps counting.  For embedders that
 * give the library a memory budget, and to exercise the out-of-memory paths
 * without exhausting a shared GPU.  Thread-safe; touches no device. */
void gx_set_device_memory_cap(uint64_t bytes);
/* Device bytes the library holds now (every allocation it made and has not
 * freed).  Thread-safe; touches no device. */
uint64_t gx_device_memory_in_use(void);

const char* gx_last_error(const gx_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GX_H */
