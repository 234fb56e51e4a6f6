// Internal declarations of the gx library (device data layouts, kernel
// parameter blocks, launchers).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gx.h"

namespace gx {

// ---------------------------------------------------------------------------
// Scene data on the device.  Triangles are regrouped into clusters of at most
// 64 triangles and 64 vertices ("meshlets") with a bounding sphere and a cone
// that bounds the face normals, so a camera can reject whole clusters that are
// outside its view or entirely back-facing before touching their triangles.
// ---------------------------------------------------------------------------
constexpr int kMeshletMaxVerts = 64;
constexpr int kMeshletMaxTris = 64;

// Five float4 per meshlet (kMeshletHdr):
//   [0] bounding sphere centre xyz, radius
//   [1] normal-cone axis xyz, sin(half angle)   (cos < -0.5 disables the test)
//   [2] cos(half angle), vertex offset (float4 units, as bits),
//       triangle offset (as bits), n_verts | n_tris << 8 (as bits)
//   [3] bounding box min xyz, min over the vertices of axis . p
//   [4] bounding box max xyz, 1 when every face normal equals the axis
//       (then the cluster is back-facing as a whole iff axis . eye <= [3].w)
constexpr int kMeshletHdr = 5;
struct DScene {
  const float4* mhdr;
  const float4* mverts;     // world positions, w unused
  const uint32_t* mtris;    // i0 | i1 << 8 | i2 << 16 (meshlet-local)
  const uint32_t* tri_rgb;  // colour per triangle, meshlet order
  int n_meshlets;
  int n_tris;
  const float* grid;        // [nz][ny][nx]
  float ox, oy, oz, h, inv_h;
  int nx, ny, nz;
  // column grid: 3 working-set radii x ncz x ncx columns, CSR offsets into
  // the free spans (lo, hi) of a sphere centre's height
  // object broad-phase lattice (four copies offset by half a cell)
  float bp_x0, bp_z0;       // corner of the unshifted grid
  int bp_nx, bp_nz;         // cells per axis of each grid
  const uint32_t* col_off;  // [3 * ncz * ncx + 1]
  const float2* col_spans;
  int ncx, ncz;
  const float* supports;    // [P][5]
  int n_supports;
  float spawn[4];
  // static distance source: 0 the dense grid above; 1 the box store, node
  // values recomputed from the solid boxes (centre xyz, -, half extents xyz,
  // - as two float4 per box) over per-cell candidate lists (cells of
  // 2^kStoreShift node intervals per axis, CSR offsets and box indices)
  int store;
  const float4* sbox;       // [n_boxes][2]
  const uint32_t* sb_off;   // [sbx * sby * sbz + 1]
  const uint16_t* sb_ids;
  int sbx, sby, sbz;
};
constexpr int kStoreShift = 4;

struct HostMeshlets {
  std::vector<float4> hdr, verts;
  std::vector<uint32_t> tris, rgb;
};

// Builds the meshlet arrays of one scene (host, deterministic).
void build_meshlets(const gx_scene_desc& s, HostMeshlets& out);

// Box store of one scene (host, deterministic; gx_store.cpp): the boxes as
// centre / half-extent float4 pairs and the CSR candidate lists per cell.
struct StoreHost {
  std::vector<float4> boxes;
  std::vector<uint32_t> off;
  std::vector<uint16_t> ids;
  int sbx = 0, sby = 0, sbz = 0;
};
bool build_box_store(const gx_scene_desc& s, StoreHost& out);

// Device robot table: gx_robot as given.
struct Robot {
  gx_robot r;
};

// Object broad-phase (appendix "Additional Collision-Detection Details"):
// per environment four regular XZ grids, cells kBpCell metres (at least
// four times the largest query radius), shifted by half a cell in x and/or
// z; a query sphere lies wholly inside one cell of one of them.  A cell
// lists up to kBpCap object indices; a fuller cell is tested by brute force.
constexpr float kBpCell = 0.5f;
constexpr int kBpCap = 12;
struct BpCell {
  uint32_t count;
  uint8_t id[kBpCap];
};
static_assert(sizeof(BpCell) == 16, "broad-phase cell");

// ---------------------------------------------------------------------------
// State: one device allocation, structure of arrays per field.
// ---------------------------------------------------------------------------
constexpr int kStateArrays = GX_STATE_ARRAYS;
struct StateView {
  float* bx;      // [n]
  float* bz;      // [n]
  float* yaw;     // [n]
  float* q;       // [7][n]
  int* held;      // [n]
  float* coff;    // [3][n]
  float* ppre;    // [3][n]
  float4* obj;    // [n][M]
  int* step;      // [n]
  int* episode;   // [n]
  float* task;    // [n][16]: goal xyz, target start xyz, previous joint actions [7],
                  // previous tip-target and target-goal distances, unused
  float4* obox;   // [n][M] box objects: half extents xyz, resting yaw (NULL: spheres)
  float* roff;    // [9][n] box objects: the held box's rotation in the tool frame
};

struct PhysicsParams {
  int n, M;
  const DScene* scenes;
  const int* env_scene;
  const Robot* robot;
  const float* actions;   // [n][11]
  StateView st;
  float* cam;             // [n][12] camera R (row-major, columns right/up/fwd) + eye
  gx_outputs out;
  unsigned* err;
  int* raster_work;       // zeroed here for the rasteriser that follows
  // neural-SDF static test: pass 1 writes the candidate sphere centres
  // (x, y, z, radius or -1 when unused) and stops; pass 2 reads the
  // predicted distances and consults the grid only below the margin.
  float4* robot_sph;                    // optional [n][32]: spheres at the accepted pose
  BpCell* bp;                           // optional [n][4][bp_cells] object broad-phase
  int bp_cells;                         // cells per grid (the largest scene's)
  int slide;                            // sliding heuristic on
  int place_jitter;                     // object placing heuristic on
  uint64_t seed;                        // Philox key (the reset key)
  int column;                           // static test on the column grid
  int nsdf_pass;                        // 0: grid only, 1: emit, 2: consume
  float4* nsdf_pts;                     // [n][32]
  const float* nsdf_d;                  // [n][32]
  float nsdf_margin;
  unsigned long long* nsdf_counters;    // optional [kNsdfCounters]
  unsigned long long* step_counters;    // optional [kStepCounters] (profile bit 4)
  int env_offset;                       // global index of environment 0 (Philox counters)
  float4* held_M;                       // box objects: [n][3] rows of the held box's world
                                        // rotation times its half extents (rasteriser)
  int store;                            // 1: scenes use the box store (kernels compiled for it)
};

// Step event counters (profile bit 4): env-steps with a contact, grasps,
// missed grasps, releases landed (also after placing jitters), releases
// restored, static and object-pair tests within kNearBand of their
// threshold, sliding moves.
enum StepCounter {
  kStepContacts = 0,
  kStepGrasps,
  kStepGraspMisses,
  kStepLanded,
  kStepRestored,
  kStepNearStatic,
  kStepNearPairs,
  kStepSlides,
  kStepCounters
};
constexpr float kNearBand = 1e-4f;  // metres

// Neural-SDF decision counters (profiling only).
enum NsdfCounter {
  kNsdfSpheres = 0,   // static tests made
  kNsdfFallbacks,     // of which the grid decided (predicted clearance < margin)
  kNsdfDisagree,      // decisions that differ from the grid-only rule
  kNsdfEnvDisagree,   // env-steps whose contact mask differs from the grid-only rule
  kNsdfCounters
};

struct ResetParams {
  BpCell* bp;          // optional broad-phase, rebuilt for each reset env
  int bp_cells;
  int n, M;
  const DScene* scenes;
  const int* env_scene;
  const Robot* robot;
  const uint8_t* mask;    // [n] or NULL
  StateView st;
  float* cam;
  uint64_t seed;
  float rho_min, rho_max;
  unsigned* err;
  int env_offset;      // global index of environment 0 (Philox counters)
  int store;           // 1: scenes use the box store (kernels compiled for it)
};

// Rasteriser launch shape: threads per CTA and CTAs wanted per SM.
constexpr int kRasterThreads = 256;
constexpr int kRasterMinBlocks = 3;

struct RasterParams {
  int n, M, W, H;
  int warps;                     // warps per CTA: 8 (0 = 8) or 12
  int big_px;                    // larger bounding boxes go to the warp scan
  unsigned long long* fb_slots;  // [n_slots][H][W] keys
  uint32_t* fb_epoch;            // [n_slots] epoch of each slot's keys (NULL: slots cleared)
  int n_slots;                   // = grid size
  int* work;                     // environment counter, zeroed before each launch
  const int* order;              // optional: k-th environment to render (costliest first)
  const DScene* scenes;
  int n_scenes;                  // env_scene values outside [0, n_scenes) are refused
  const int* env_scene;
  const float* cam;        // [n][12]
  const float4* obj;       // [n][M]
  const float4* omesh_v;   // [nv] unit instance mesh
  const uint32_t* omesh_t; // [nt] packed
  int omesh_nv, omesh_nt;
  const uint32_t* obj_rgb; // [GX_MAX_OBJECTS objects + 32 robot spheres]
  const float4* robot_sph; // optional [n][32] robot sphere centre, radius (0: unused)
  const float4* obox;      // box objects: [n][M] half extents, yaw (NULL: spheres)
  const float4* held_M;    // box objects: [n][3] the held box's world rotation x extents
  const int* held;         // box objects: [n] held object index
  uint32_t* vis;           // occlusion culling: [n][vis_words] clusters shown in the last image
  int vis_words;
  float near_;
  void* depth;
  int depth_fp16;
  uint8_t* rgb;
  unsigned* err;
  unsigned long long* counters;  // optional [kRasterCounters] work counters
};

// Rasteriser work counters (profiling only).
enum RasterCounter {
  kCntClustersTested = 0,
  kCntClustersDrawn,
  kCntTrisSeen,
  kCntTrisFront,
  kCntTrisSmall,
  kCntSmallPixels,
  kCntTrisBig,
  kCntBigBlocks,
  kCntTrisClipped,
  kCntFragments,
  kCntWaitIters,     // mbarrier polls (per warp)
  kCntExpandTrips,   // fragment-expansion loop trips (per warp)
  kCntRounds,        // 32-triangle rounds (per warp)
  kCntExpandSlots,   // fragment-expansion slots (runs of up to four pixels)
  kCntClustersOccluded,  // clusters skipped by the occlusion test
  kRasterCounters
};

void launch_physics(const PhysicsParams& p, cudaStream_t s);        // dispatches on p.store
void launch_physics_store(const PhysicsParams& p, cudaStream_t s);  // box-store kernels
void launch_reset_store(const ResetParams& p, cudaStream_t s);
cudaError_t reset_configure_store();
void launch_bp_rebuild(const DScene* scenes, const int* env_scene, const StateView& st, int n,
                       int M, BpCell* bp, int cells, cudaStream_t s);
void launch_reset(const ResetParams& p, cudaStream_t s);
void launch_physics_boxes(const PhysicsParams& p, cudaStream_t s);

// One persistent cooperative launch per step: masked resets, physics and
// rendering separated by grid-wide barriers (gx_fused.cu).
constexpr int kFusedResetScratch = 2376;  // float4 per CTA: the reset's try table and objects
struct FusedParams {
  PhysicsParams pp;
  ResetParams rs;
  RasterParams rp;
  const uint8_t* reset_mask;  // NULL: no reset phase
  float4* reset_scratch;      // [ctas][kFusedResetScratch]
  float4* obj_scratch;        // [ctas][8 warps][GX_MAX_OBJECTS] objects of physics (> 128 objects)
  unsigned* barrier;          // [2] arrivals (zeroed before each launch), generation
};
cudaError_t fused_configure();
cudaError_t fused_max_ctas(int* ctas);
cudaError_t launch_fused_step(const FusedParams& f, int ctas, cudaStream_t s);
void launch_reset_boxes(const ResetParams& p, cudaStream_t s);         // dispatches on p.store
void launch_physics_boxes_store(const PhysicsParams& p, cudaStream_t s);  // box-store kernels
void launch_reset_boxes_store(const ResetParams& p, cudaStream_t s);
cudaError_t reset_configure();
void launch_raster(const RasterParams& p, cudaStream_t s);
// ---------------------------------------------------------------------------
// Neural SDF of one scene (Fourier-feature MLP 64 -> 128 x4 -> 1).
// ---------------------------------------------------------------------------
constexpr int kNsdfFreq = 32;    // Fourier frequencies (64 features)
constexpr int kNsdfWidth = 128;  // hidden width
constexpr int kNsdfParams = 128 * 64 + 128 + 3 * (128 * 128 + 128) + 128 + 1;  // 57,985
// Device blob read by the kernels: BF16 weight images laid out exactly as
// the tensor cores read them from shared memory (K-major, 128-byte swizzle),
// then FP32 biases, the FP32 output row and the Fourier matrix.
constexpr int kNsdfW1Bytes = 128 * 64 * 2;    // 16 KB
constexpr int kNsdfWhBytes = 128 * 128 * 2;   // 32 KB each for layers 2..4
constexpr int kNsdfImgBytes = kNsdfW1Bytes + 3 * kNsdfWhBytes;  // 112 KB
struct NsdfTail {            // follows the weight images in the blob
  float b[4][128];           // hidden biases
  float w5[128];             // output row
  float b5;
  float centre[3];           // features use x - centre
  float B[kNsdfFreq][3];     // Fourier matrix
  float pad[4];
};
constexpr int kNsdfBlobBytes = kNsdfImgBytes + (int)sizeof(NsdfTail);
struct NsdfScene {
  unsigned char* blob = nullptr;  // device, kNsdfBlobBytes
  float* master = nullptr;        // device FP32 parameters (kNsdfParams), training only
  bool ready = false;
};

}  // namespace gx

struct gx_scene_set {
  int n = 0;
  std::vector<gx::DScene> host;
  gx::DScene* d_scenes = nullptr;     // default view: dense grid when built, else box store
  gx::DScene* d_scenes_box = nullptr; // the same scenes with the box store
  bool dense = true;                  // dense grids built
  bool columns = true;                // column grids built
  std::vector<size_t> dense_bytes, store_bytes, render_bytes;
  std::vector<void*> allocs;
  float4* omesh_v = nullptr;
  uint32_t* omesh_t = nullptr;
  uint32_t* obj_rgb = nullptr;
  int omesh_nv = 0, omesh_nt = 0;
  std::vector<int> meshlets_per_scene;
  std::vector<gx::NsdfScene> nsdf;
  std::vector<size_t> column_bytes;  // column grid size per scene
  int device = -1;                   // CUDA device current at creation (holds every buffer)
};

namespace gx {

void nsdf_free(gx_scene_set* s);

// Neural-SDF queries of a step: tiles of up to 4 environments (128 rows of
// 32 sphere slots) that share a scene.
struct NsdfStepParams {
  const unsigned char* const* blobs;  // [n_scenes] device blob per scene
  const int4* tiles;                  // (scene, first index into perm, count, 0)
  int n_tiles;
  const int* perm;                    // environments grouped by scene
  const float4* pts;                  // [n][32]
  float* out;                         // [n][32]
  unsigned* err;
};
cudaError_t nsdf_launch_step(const NsdfStepParams& p, cudaStream_t s);

// Read-only view of a scene set's device data, for entry points outside
// gx_api.cu.
struct SceneSetView {
  const DScene* scenes;
  int n;
  const float4* omesh_v;
  const uint32_t* omesh_t;
  int omesh_nv, omesh_nt;
  const uint32_t* obj_rgb;
  int device;                         // CUDA device holding the set's buffers
};
bool scene_set_view(const gx_scene_set* set, SceneSetView* out);
gx_status set_last_error(gx_status s, const char* msg);

// Column grid constants (working-set radii, spacing, per-column interval cap).
constexpr double kColumnSpacing = 0.03;
constexpr int kColumnCap = 64;
__device__ constexpr double kColumnRadius[3] = {0.015, 0.05, 0.12};
void launch_column_build(const float* boxes, int n_boxes, double ox, double oz, double ylo,
                         double yhi, int ncx, int ncz, const uint32_t* offsets, uint32_t* counts,
                         float2* spans, unsigned* overflow, cudaStream_t s);

size_t raster_smem_bytes(int warps = 8, int hiz_tiles = 0);
cudaError_t raster_configure(int* slots);
// resident rasteriser CTAs per SM of a shape (boxes: the box-object kernel)
cudaError_t raster_ctas_per_sm(int warps, int* per_sm, bool boxes = false);
void launch_grid_build(float* grid, const float* boxes, int n_boxes, float ox, float oy, float oz,
                       float h, int nx, int ny, int nz, cudaStream_t s);
// Trilinear static distance of scene `scene` at n points (NaN outside the box).
cudaError_t launch_static_distance(const DScene* scenes, int scene, const float* pts, int n,
                                   float* dist, cudaStream_t s);

// Device allocations of the library: cudaMalloc / cudaFree with the bytes
// counted against the optional cap of gx_set_device_memory_cap (an
// allocation past it fails with cudaErrorMemoryAllocation, which every
// caller maps to GX_ENOMEM).
cudaError_t dev_malloc_bytes(void** p, size_t bytes);
void dev_free(void* p);
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_bytes(reinterpret_cast<void**>(p), bytes);
}

// device error bits beyond the public ones
constexpr unsigned kErrWaitTimeout = 0x100u;  // a bounded mbarrier wait gave up
constexpr unsigned kErrBadScene = 0x200u;     // a scene index outside the set (env drawn empty)

}  // namespace gx
