// Host implementation of the C ABI declared in include/gx.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gx_internal.h"

using namespace gx;

namespace {

thread_local std::string g_last_error;

// An NVTX range over the rest of the scope when `on` (profile bit 3): marks a
// call's host enqueue for timeline and ncu --nvtx filtering.
struct NvtxRange {
  bool on;
  NvtxRange(bool o, const char* name) : on(o) {
    if (on) nvtxRangePushA(name);
  }
  ~NvtxRange() {
    if (on) nvtxRangePop();
  }
};

// Device bytes the library holds, per allocation, and the optional cap.
std::mutex g_mem_mu;
std::unordered_map<void*, size_t> g_mem_sizes;
uint64_t g_mem_in_use = 0, g_mem_cap = 0;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace


struct gx_ctx {
  const gx_scene_set* set = nullptr;
  const DScene* scenes = nullptr;      // the set's scenes with this context's static store
  gx_config cfg{};
  int n = 0, M = 0, big_px = 0, n_slots = 0;
  int raster_ctas = 0;                 // CTAs launched (<= n_slots), set by the autotuner
  int raster_warps = 8;                // warps per rasteriser CTA (6, 7, 8 or 12)
  int slots8 = 0;                      // resident 8-warp rasteriser CTAs (<= n_slots)
  int per_sm6 = 0;                     // resident 6-warp CTAs per SM (0: shape not offered)
  int per_sm7 = 0;                     // resident 7-warp CTAs per SM (0: shape not offered)
  int order_mode = 0;                  // 0: index order, 1: costliest scene first
  int* d_order = nullptr;              // environments, costliest scene first
  int sms = 0;
  unsigned long long* d_fb = nullptr;  // rasteriser framebuffer slots
  uint32_t* d_fb_epoch = nullptr;      // epoch of each slot's keys
  int* d_raster_work = nullptr;
  float near_ = 0.05f;
  Robot* d_robot = nullptr;
  int* d_env_scene = nullptr;
  void* d_state = nullptr;
  size_t state_bytes = 0;
  size_t off[kStateArrays] = {0};
  StateView st{};
  float* d_cam = nullptr;
  float4* d_robot_sph = nullptr;       // robot spheres for rendering the robot body
  float4* d_held_M = nullptr;          // box objects: the held box's world rotation x extents
  uint32_t* d_vis = nullptr;           // occlusion culling: clusters shown in the last image
  int vis_words = 0;
  bool occlusion = false;              // occlusion culling in use (the autotuner may change it)
  // fused step (one cooperative launch per step)
  int fused_ctas = 0;
  float4* d_fused_scratch = nullptr;   // reset try tables, per CTA
  float4* d_fused_obj = nullptr;       // physics object copies above 128 objects, per CTA
  unsigned* d_barrier = nullptr;       // grid barrier: arrivals, generation
  cudaError_t launch_err = cudaSuccess;
  const uint8_t* g_mask = nullptr;     // reset mask captured in the graph (gx_step_reset)
  BpCell* d_bp = nullptr;              // object broad-phase cells
  int bp_cells = 0;
  unsigned* d_err = nullptr;
  unsigned long long* d_step_counters = nullptr;  // profile bit 4: step event counters
  unsigned* h_err = nullptr;
  cudaEvent_t ev_err = nullptr;
  bool err_pending = false;
  unsigned dev_err_seen = 0;
  std::string msg;
  // graph replay
  cudaGraphExec_t gexec = nullptr;
  const float* g_actions = nullptr;
  gx_outputs g_out{};
  // profiling: event triples per timed launch group, read back lazily
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_kind;   // 0 = step, 1 = reset, 2 = step with neural-SDF queries
  std::vector<size_t> prof_at;  // first event of each group
  size_t prof_used = 0;
  double prof_ms[4] = {0, 0, 0, 0};
  int64_t prof_n[4] = {0, 0, 0, 0};
  unsigned long long* d_counters = nullptr;
  // neural SDF in the static test
  float4* d_nsdf_pts = nullptr;
  float* d_nsdf_d = nullptr;
  int4* d_nsdf_tiles = nullptr;
  int n_nsdf_tiles = 0;
  int* d_nsdf_perm = nullptr;
  const unsigned char** d_nsdf_blobs = nullptr;
  unsigned long long* d_nsdf_counters = nullptr;
  // buffers for gx_step_host
  float* h2d_actions = nullptr;
  gx_outputs dev_out{};
  std::vector<void*> host_step_allocs;
};

namespace {

gx_status fail(gx_ctx* c, gx_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->msg = buf;
  g_last_error = buf;
  return s;
}

#define CK(ctx, call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? GX_ENOMEM : GX_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                         \
  } while (0)

}  // namespace

cudaError_t gx::dev_malloc_bytes(void** p, size_t bytes) {
  *p = nullptr;
  std::lock_guard<std::mutex> lock(g_mem_mu);
  if (g_mem_cap && g_mem_in_use + bytes > g_mem_cap) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  g_mem_sizes[*p] = bytes;
  g_mem_in_use += bytes;
  return cudaSuccess;
}

void gx::dev_free(void* p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lock(g_mem_mu);
    auto it = g_mem_sizes.find(p);
    if (it != g_mem_sizes.end()) {
      g_mem_in_use -= it->second;
      g_mem_sizes.erase(it);
    }
  }
  cudaFree(p);
}

extern "C" void gx_set_device_memory_cap(uint64_t bytes) {
  std::lock_guard<std::mutex> lock(g_mem_mu);
  g_mem_cap = bytes;
}

extern "C" uint64_t gx_device_memory_in_use(void) {
  std::lock_guard<std::mutex> lock(g_mem_mu);
  return g_mem_in_use;
}

namespace {

template <class T>
cudaError_t upload(gx_scene_set* s, T** dst, const T* src, size_t count) {
  *dst = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = dev_malloc((void**)dst, count * sizeof(T));
  if (e != cudaSuccess) return e;
  s->allocs.push_back(*dst);
  return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

void free_set(gx_scene_set* s) {
  if (!s) return;
  for (void* p : s->allocs) dev_free(p);
  nsdf_free(s);
  delete s;
}

// Reads the device error word if its asynchronous copy has landed.
gx_status poll_device_error(gx_ctx* c, bool wait) {
  if (!c->err_pending) return GX_OK;
  if (wait) {
    if (cudaEventSynchronize(c->ev_err) != cudaSuccess)
      return fail(c, GX_ECUDA, "cudaEventSynchronize failed");
  } else if (cudaEventQuery(c->ev_err) != cudaSuccess) {
    return GX_OK;
  }
  c->err_pending = false;
  const unsigned v = *c->h_err;
  if (v) {
    *c->h_err = 0;
    c->dev_err_seen |= v;
    cudaMemset(c->d_err, 0, sizeof(unsigned));
    // a crowded reset keeping an object's last try is reported by
    // gx_device_error but does not fail the call
    if ((v & ~GX_DEV_PLACEMENT_FAILED) == 0) return GX_OK;
    return fail(c, GX_EDEVICE, "device error word 0x%x:%s%s%s%s", v,
                (v & GX_DEV_NONFINITE_ACTION) ? " non-finite action (used 0)" : "",
                (v & GX_DEV_PLACEMENT_FAILED) ? " reset placement used all tries" : "",
                (v & kErrWaitTimeout) ? " bounded wait gave up" : "",
                (v & kErrBadScene) ? " scene index out of range" : "");
  }
  return GX_OK;
}

gx_status post_error_copy(gx_ctx* c, cudaStream_t s) {
  CK(c, cudaMemcpyAsync(c->h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(c, cudaEventRecord(c->ev_err, s));
  c->err_pending = true;
  return GX_OK;
}

bool same_outputs(const gx_outputs& a, const gx_outputs& b) {
  return std::memcmp(&a, &b, sizeof(gx_outputs)) == 0;
}

// Events for the next timed launch group: 5 for a step (start, after
// physics pass 1, after the neural-SDF queries, after physics, after the
// rasteriser), 2 for a reset.  nullptr once the pool is full;
// gx_phase_times drains it.
cudaEvent_t* prof_slot(gx_ctx* c, int kind) {
  const size_t kMax = 5 * 8192, k = (kind == 1 || kind == 3) ? 2 : 5;
  if (c->prof_used + k > kMax) return nullptr;
  while (c->prof_ev.size() < c->prof_used + k) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->prof_ev.push_back(e);
  }
  c->prof_kind.push_back(kind);
  c->prof_at.push_back(c->prof_used);
  cudaEvent_t* r = &c->prof_ev[c->prof_used];
  c->prof_used += k;
  return r;
}

PhysicsParams physics_params(gx_ctx* c, const float* actions, const gx_outputs& out) {
  PhysicsParams pp{};
  pp.n = c->n;
  pp.M = c->M;
  pp.scenes = c->scenes;
  pp.env_scene = c->d_env_scene;
  pp.robot = c->d_robot;
  pp.actions = actions;
  pp.st = c->st;
  pp.cam = c->d_cam;
  pp.robot_sph = c->d_robot_sph;
  pp.bp = c->d_bp;
  pp.bp_cells = c->bp_cells;
  pp.out = out;
  pp.err = c->d_err;
  pp.raster_work = c->d_raster_work;
  pp.slide = c->cfg.heuristics & 1;
  pp.place_jitter = (c->cfg.heuristics >> 1) & 1;
  pp.seed = c->cfg.seed;
  pp.env_offset = c->cfg.env_offset;
  pp.column = c->cfg.sdf_mode == 2;
  pp.store = c->cfg.static_store;
  pp.step_counters = c->d_step_counters;
  return pp;
}

RasterParams raster_params(gx_ctx* c, const gx_outputs& out) {
  RasterParams rp{};
  rp.n = c->n;
  rp.M = c->M;
  rp.W = c->cfg.img_w;
  rp.H = c->cfg.img_h;
  rp.warps = c->cfg.fused_step ? 8 : c->raster_warps;
  rp.big_px = c->big_px;
  rp.fb_slots = c->d_fb;
  rp.fb_epoch = c->d_fb_epoch;
  rp.n_slots = c->raster_ctas;
  rp.order = c->order_mode ? c->d_order : nullptr;
  rp.work = c->d_raster_work;
  rp.scenes = c->scenes;
  rp.n_scenes = c->set->n;
  rp.env_scene = c->d_env_scene;
  rp.cam = c->d_cam;
  rp.obj = c->st.obj;
  rp.omesh_v = c->set->omesh_v;
  rp.omesh_t = c->set->omesh_t;
  rp.omesh_nv = c->set->omesh_nv;
  rp.omesh_nt = c->set->omesh_nt;
  rp.obj_rgb = c->set->obj_rgb;
  rp.robot_sph = c->d_robot_sph;
  if (c->occlusion && !c->cfg.fused_step && !c->cfg.object_boxes) {
    rp.vis = c->d_vis;
    rp.vis_words = c->vis_words;
  }
  if (c->cfg.object_boxes) {
    rp.obox = c->st.obox;
    rp.held_M = c->d_held_M;
    rp.held = c->st.held;
  }
  rp.near_ = c->near_;
  rp.depth = out.depth;
  rp.depth_fp16 = c->cfg.depth_fp16;
  rp.rgb = c->cfg.render_rgb ? out.rgb : nullptr;
  rp.err = c->d_err;
  rp.counters = (c->cfg.profile & 2) ? c->d_counters : nullptr;
  return rp;
}

ResetParams reset_params(gx_ctx* x, const uint8_t* env_mask) {
  ResetParams rp{};
  rp.n = x->n;
  rp.M = x->M;
  rp.scenes = x->scenes;
  rp.env_scene = x->d_env_scene;
  rp.robot = x->d_robot;
  rp.mask = env_mask;
  rp.st = x->st;
  rp.cam = x->d_cam;
  rp.seed = x->cfg.seed;
  rp.env_offset = x->cfg.env_offset;
  rp.rho_min = x->cfg.obj_radius_min;
  rp.rho_max = x->cfg.obj_radius_max;
  rp.err = x->d_err;
  rp.bp = x->d_bp;
  rp.bp_cells = x->bp_cells;
  rp.store = x->cfg.static_store;
  return rp;
}

void enqueue_step(gx_ctx* c, const float* actions, const gx_outputs& out, cudaStream_t s) {
  const bool nvtx = (c->cfg.profile & 8) != 0;
  const bool neural = c->cfg.sdf_mode == 1;
  cudaEvent_t* ev = (c->cfg.profile & 1) ? prof_slot(c, neural ? 2 : 0) : nullptr;
  if (ev) cudaEventRecord(ev[0], s);
  PhysicsParams pp = physics_params(c, actions, out);
  if (c->cfg.sdf_mode == 1) {
    pp.nsdf_pts = c->d_nsdf_pts;
    pp.nsdf_d = c->d_nsdf_d;
    pp.nsdf_margin = c->cfg.sdf_margin;
    pp.nsdf_counters = (c->cfg.profile & 4) ? c->d_nsdf_counters : nullptr;
    pp.nsdf_pass = 1;
    {
      NvtxRange r(nvtx, "gx physics pass 1");
      launch_physics(pp, s);
    }
    if (ev) cudaEventRecord(ev[1], s);
    NsdfStepParams np{};
    np.blobs = c->d_nsdf_blobs;
    np.tiles = c->d_nsdf_tiles;
    np.n_tiles = c->n_nsdf_tiles;
    np.perm = c->d_nsdf_perm;
    np.pts = c->d_nsdf_pts;
    np.out = c->d_nsdf_d;
    np.err = c->d_err;
    {
      NvtxRange r(nvtx, "gx neural-SDF queries");
      nsdf_launch_step(np, s);
    }
    if (ev) cudaEventRecord(ev[2], s);
    pp.nsdf_pass = 2;
  }
  {
    NvtxRange r(nvtx, "gx physics");
    if (c->cfg.object_boxes) {
      pp.held_M = c->d_held_M;
      launch_physics_boxes(pp, s);
    } else {
      launch_physics(pp, s);
    }
  }
  if (ev) cudaEventRecord(ev[3], s);
  {
    NvtxRange r(nvtx, "gx raster");
    launch_raster(raster_params(c, out), s);
  }
  if (ev) cudaEventRecord(ev[4], s);
}

// The fused step: masked resets (mask may be NULL), physics and rendering in
// one cooperative launch; the barrier's arrival count is cleared first.
void enqueue_fused(gx_ctx* c, const uint8_t* mask, const float* actions, const gx_outputs& out,
                   cudaStream_t s) {
  cudaEvent_t* ev = (c->cfg.profile & 1) ? prof_slot(c, 3) : nullptr;
  FusedParams f{};
  f.pp = physics_params(c, actions, out);
  f.pp.raster_work = nullptr;
  f.rs = reset_params(c, mask);
  f.rp = raster_params(c, out);
  f.reset_mask = mask;
  f.reset_scratch = c->d_fused_scratch;
  f.obj_scratch = c->d_fused_obj;
  f.barrier = c->d_barrier;
  cudaMemsetAsync(c->d_barrier, 0, sizeof(unsigned), s);
  if (ev) cudaEventRecord(ev[0], s);
  cudaError_t e = launch_fused_step(f, std::min(c->fused_ctas, c->raster_ctas), s);
  if (e != cudaSuccess) c->launch_err = e;
  if (ev) cudaEventRecord(ev[1], s);
}

}  // namespace

// ===========================================================================
// scene sets
// ===========================================================================
extern "C" gx_status gx_scene_set_create(const gx_scene_desc* scenes, int32_t n_scenes,
                                         const gx_object_mesh* mesh, gx_scene_set** out) {
  gx_scene_options opt{};
  opt.dense_grid = 1;
  opt.column_grid = 1;
  return gx_scene_set_create_ex(scenes, n_scenes, mesh, &opt, out);
}

extern "C" gx_status gx_scene_set_create_ex(const gx_scene_desc* scenes, int32_t n_scenes,
                                            const gx_object_mesh* mesh,
                                            const gx_scene_options* opt, gx_scene_set** out) {
  if (!out) return fail(nullptr, GX_EINVAL, "gx_scene_set_create: out is NULL");
  *out = nullptr;
  if (!opt || (opt->dense_grid != 0 && opt->dense_grid != 1) ||
      (opt->column_grid != 0 && opt->column_grid != 1))
    return fail(nullptr, GX_EINVAL, "scene options: dense_grid and column_grid must be 0 or 1");
  if (!scenes || n_scenes < 1) return fail(nullptr, GX_EINVAL, "need at least one scene");
  if (!mesh || mesh->n_verts < 1 || mesh->n_verts > 32 || mesh->n_tris < 1 ||
      mesh->n_tris > 32 || !mesh->verts || !mesh->tris)
    return fail(nullptr, GX_EINVAL, "object mesh must have 1..32 vertices and triangles");
  for (int i = 0; i < n_scenes; ++i) {
    const gx_scene_desc& d = scenes[i];
    if (d.n_boxes < 1 || !d.boxes || d.n_boxes > 4096)
      return fail(nullptr, GX_EINVAL, "scene %d: need 1..4096 boxes", i);
    if (d.n_tris < 0 || (d.n_tris > 0 && (!d.verts || !d.tris || !d.tri_rgb)) || d.n_verts < 0)
      return fail(nullptr, GX_EINVAL, "scene %d: bad triangle arrays", i);
    for (int t = 0; t < 3 * d.n_tris; ++t)
      if (d.tris[t] < 0 || d.tris[t] >= d.n_verts)
        return fail(nullptr, GX_EINVAL, "scene %d: triangle index out of range", i);
    if (d.n_supports < 1 || !d.supports) return fail(nullptr, GX_EINVAL, "scene %d: no supports", i);
    if (!(d.grid_h > 0.f) || d.grid_dims[0] < 2 || d.grid_dims[1] < 2 || d.grid_dims[2] < 2)
      return fail(nullptr, GX_EINVAL, "scene %d: bad grid", i);
    if ((double)d.grid_dims[0] * d.grid_dims[1] * d.grid_dims[2] > 2.0e9)
      return fail(nullptr, GX_EINVAL, "scene %d: grid too large", i);
  }
  for (int t = 0; t < 3 * mesh->n_tris; ++t)
    if (mesh->tris[t] < 0 || mesh->tris[t] >= mesh->n_verts)
      return fail(nullptr, GX_EINVAL, "object mesh: index out of range");

  gx_scene_set* s = new gx_scene_set();
  s->n = n_scenes;
  s->host.resize(n_scenes);
  s->dense = opt->dense_grid == 1;
  s->columns = opt->column_grid == 1;
  auto bail = [&](cudaError_t e, const char* what) {
    free_set(s);
    return fail(nullptr, e == cudaErrorMemoryAllocation ? GX_ENOMEM : GX_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&s->device)) != cudaSuccess) return bail(e, "current device");
  for (int i = 0; i < n_scenes; ++i) {
    const gx_scene_desc& d = scenes[i];
    DScene& ds = s->host[i];
    HostMeshlets hm;
    build_meshlets(d, hm);
    s->meshlets_per_scene.push_back((int)(hm.hdr.size() / kMeshletHdr));
    if (hm.verts.size() >= (1u << 24) || hm.tris.size() >= (1u << 24)) {
      free_set(s);
      return fail(nullptr, GX_EINVAL, "scene %d: more than 2^24 cluster vertices or triangles", i);
    }
    if ((e = upload(s, (float4**)&ds.mhdr, hm.hdr.data(), hm.hdr.size())) != cudaSuccess)
      return bail(e, "upload meshlets");
    if ((e = upload(s, (float4**)&ds.mverts, hm.verts.data(), hm.verts.size())) != cudaSuccess)
      return bail(e, "upload vertices");
    if ((e = upload(s, (uint32_t**)&ds.mtris, hm.tris.data(), hm.tris.size())) != cudaSuccess)
      return bail(e, "upload triangles");
    if ((e = upload(s, (uint32_t**)&ds.tri_rgb, hm.rgb.data(), hm.rgb.size())) != cudaSuccess)
      return bail(e, "upload colours");
    ds.n_meshlets = (int)(hm.hdr.size() / kMeshletHdr);
    ds.n_tris = (int)hm.tris.size();
    if ((e = upload(s, (float**)&ds.supports, d.supports, (size_t)5 * d.n_supports)) != cudaSuccess)
      return bail(e, "upload supports");
    ds.n_supports = d.n_supports;
    ds.ox = d.grid_origin[0];
    ds.oy = d.grid_origin[1];
    ds.oz = d.grid_origin[2];
    ds.h = d.grid_h;
    ds.inv_h = 1.0f / d.grid_h;
    ds.nx = d.grid_dims[0];
    ds.ny = d.grid_dims[1];
    ds.nz = d.grid_dims[2];
    for (int k = 0; k < 4; ++k) ds.spawn[k] = d.spawn[k];
    s->render_bytes.push_back((hm.hdr.size() + hm.verts.size()) * sizeof(float4) +
                              (hm.tris.size() + hm.rgb.size()) * sizeof(uint32_t));
    const size_t nodes = (size_t)ds.nx * ds.ny * ds.nz;
    float* dboxes = nullptr;
    if ((e = upload(s, &dboxes, d.boxes, (size_t)6 * d.n_boxes)) != cudaSuccess)
      return bail(e, "upload boxes");
    ds.grid = nullptr;
    if (s->dense) {
      float* grid = nullptr;
      if ((e = dev_malloc(&grid, nodes * sizeof(float))) != cudaSuccess) return bail(e, "grid");
      s->allocs.push_back(grid);
      launch_grid_build(grid, dboxes, d.n_boxes, ds.ox, ds.oy, ds.oz, ds.h, ds.nx, ds.ny, ds.nz, 0);
      if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "grid kernel");
      ds.grid = grid;
    }
    s->dense_bytes.push_back(s->dense ? nodes * sizeof(float) : 0);
    {
      // box store: boxes and per-cell candidate lists (the kernels pick it
      // per context; see gx_config.static_store)
      StoreHost sh;
      if (!build_box_store(d, sh)) {
        free_set(s);
        return fail(nullptr, GX_EINVAL, "scene %d: box store too large", i);
      }
      if ((e = upload(s, (float4**)&ds.sbox, sh.boxes.data(), sh.boxes.size())) != cudaSuccess ||
          (e = upload(s, (uint32_t**)&ds.sb_off, sh.off.data(), sh.off.size())) != cudaSuccess)
        return bail(e, "upload box store");
      if (!sh.ids.empty() &&
          (e = upload(s, (uint16_t**)&ds.sb_ids, sh.ids.data(), sh.ids.size())) != cudaSuccess)
        return bail(e, "upload box store");
      ds.sbx = sh.sbx;
      ds.sby = sh.sby;
      ds.sbz = sh.sbz;
      ds.store = 0;
      s->store_bytes.push_back(sh.boxes.size() * sizeof(float4) + sh.off.size() * 4 +
                               sh.ids.size() * 2);
    }
    // object broad-phase lattice: the grid box with a cell of margin
    ds.bp_x0 = ds.ox - kBpCell;
    ds.bp_z0 = ds.oz - kBpCell;
    ds.bp_nx = (int)std::ceil(((ds.nx - 1) * (double)ds.h + 2 * kBpCell) / kBpCell) + 1;
    ds.bp_nz = (int)std::ceil(((ds.nz - 1) * (double)ds.h + 2 * kBpCell) / kBpCell) + 1;
    if (!s->columns) {
      ds.ncx = ds.ncz = 0;
      ds.col_off = nullptr;
      ds.col_spans = nullptr;
      s->column_bytes.push_back(0);
    } else {
      // column grid over the same box: count, prefix sum on the host, fill
      const double h = (double)ds.h;
      ds.ncx = (int)std::floor((ds.nx - 1) * h / kColumnSpacing + 1e-6) + 1;
      ds.ncz = (int)std::floor((ds.nz - 1) * h / kColumnSpacing + 1e-6) + 1;
      const size_t ncol = (size_t)3 * ds.ncx * ds.ncz;
      const double ylo = (double)ds.oy, yhi = ylo + (ds.ny - 1) * h;
      uint32_t *cnt = nullptr, *off = nullptr;
      unsigned* ovf = nullptr;
      float2* spans = nullptr;
      if ((e = dev_malloc(&cnt, ncol * 4)) != cudaSuccess) return bail(e, "columns");
      s->allocs.push_back(cnt);
      if ((e = dev_malloc(&ovf, 4)) != cudaSuccess) return bail(e, "columns");
      s->allocs.push_back(ovf);
      cudaMemset(ovf, 0, 4);
      launch_column_build(dboxes, d.n_boxes, (double)ds.ox, (double)ds.oz, ylo, yhi, ds.ncx, ds.ncz,
                          nullptr, cnt, nullptr, ovf, 0);
      std::vector<uint32_t> hc(ncol);
      if ((e = cudaMemcpy(hc.data(), cnt, ncol * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return bail(e, "column counts");
      std::vector<uint32_t> ho(ncol + 1);
      uint64_t acc = 0;
      for (size_t c = 0; c < ncol; ++c) {
        ho[c] = (uint32_t)acc;
        acc += hc[c];
      }
      ho[ncol] = (uint32_t)acc;
      if (acc >= ((uint64_t)1 << 32)) {
        free_set(s);
        return fail(nullptr, GX_EINVAL, "scene %d: too many column spans", i);
      }
      if ((e = upload(s, &off, ho.data(), ho.size())) != cudaSuccess) return bail(e, "columns");
      if ((e = dev_malloc(&spans, (acc ? acc : 1) * sizeof(float2))) != cudaSuccess)
        return bail(e, "column spans");
      s->allocs.push_back(spans);
      launch_column_build(dboxes, d.n_boxes, (double)ds.ox, (double)ds.oz, ylo, yhi, ds.ncx, ds.ncz,
                          off, cnt, spans, ovf, 0);
      unsigned hovf = 0;
      if ((e = cudaMemcpy(&hovf, ovf, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return bail(e, "column build");
      if (hovf) {
        free_set(s);
        return fail(nullptr, GX_EINVAL, "scene %d: a column meets more than %d boxes", i,
                    kColumnCap);
      }
      ds.col_off = off;
      ds.col_spans = spans;
      s->column_bytes.push_back((ncol + 1) * 4 + acc * sizeof(float2));
    }
  }
  std::vector<float4> ov(mesh->n_verts);
  for (int k = 0; k < mesh->n_verts; ++k)
    ov[k] = make_float4(mesh->verts[3 * k], mesh->verts[3 * k + 1], mesh->verts[3 * k + 2], 0.f);
  std::vector<uint32_t> ot(mesh->n_tris);
  for (int t = 0; t < mesh->n_tris; ++t)
    ot[t] = (uint32_t)mesh->tris[3 * t] | ((uint32_t)mesh->tris[3 * t + 1] << 8) |
            ((uint32_t)mesh->tris[3 * t + 2] << 16);
  if ((e = upload(s, &s->omesh_v, ov.data(), ov.size())) != cudaSuccess) return bail(e, "mesh");
  if ((e = upload(s, &s->omesh_t, ot.data(), ot.size())) != cudaSuccess) return bail(e, "mesh");
  std::vector<uint32_t> rgb96(GX_MAX_OBJECTS + 32);
  std::memcpy(rgb96.data(), mesh->obj_rgb, GX_MAX_OBJECTS * 4);
  std::memcpy(rgb96.data() + GX_MAX_OBJECTS, mesh->robot_rgb, 32 * 4);
  if ((e = upload(s, &s->obj_rgb, rgb96.data(), rgb96.size())) != cudaSuccess)
    return bail(e, "colours");
  s->omesh_nv = mesh->n_verts;
  s->omesh_nt = mesh->n_tris;
  std::vector<DScene> boxed = s->host;
  for (DScene& ds : boxed) ds.store = 1;
  if ((e = upload(s, &s->d_scenes_box, boxed.data(), boxed.size())) != cudaSuccess)
    return bail(e, "scene table");
  if (s->dense) {
    if ((e = upload(s, &s->d_scenes, s->host.data(), s->host.size())) != cudaSuccess)
      return bail(e, "scene table");
  } else {
    s->host = boxed;
    s->d_scenes = s->d_scenes_box;
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(e, "scene build");
  *out = s;
  return GX_OK;
}

extern "C" gx_status gx_scene_set_destroy(gx_scene_set* set) {
  free_set(set);
  return GX_OK;
}

// ===========================================================================
// contexts
// ===========================================================================
extern "C" gx_status gx_create(const gx_scene_set* set, const gx_robot* robot,
                               const gx_config* cfg, gx_ctx** out) {
  if (!out) return fail(nullptr, GX_EINVAL, "gx_create: out is NULL");
  *out = nullptr;
  if (!set || !robot || !cfg) return fail(nullptr, GX_EINVAL, "gx_create: NULL argument");
  const gx_config& c = *cfg;
  if (c.n_envs < 1) return fail(nullptr, GX_EINVAL, "n_envs must be >= 1");
  if (c.img_w < 32 || c.img_h < 32 || c.img_w > 256 || c.img_h > 256 || c.img_w % 32 ||
      c.img_h % 32)
    return fail(nullptr, GX_EINVAL, "image sides must be multiples of 32 in [32, 256]");
  if (c.n_objects < 0 || c.n_objects > GX_MAX_OBJECTS)
    return fail(nullptr, GX_EINVAL, "n_objects must be in [0, 256]");
  if (!(c.obj_radius_min > 0.f) || !(c.obj_radius_max >= c.obj_radius_min))
    return fail(nullptr, GX_EINVAL, "bad object radius range");
  if (robot->n_spheres < 1 || robot->n_spheres > 30)
    return fail(nullptr, GX_EINVAL, "robot needs 1..30 spheres");
  for (int i = 0; i < robot->n_spheres; ++i)
    if (robot->sphere_link[i] < 0 || robot->sphere_link[i] > 7 || !(robot->sphere_radius[i] > 0.f))
      return fail(nullptr, GX_EINVAL, "robot sphere %d: bad link or radius", i);
  for (int k = 0; k < 7; ++k)
    if (robot->link_axis[k] < 0 || robot->link_axis[k] > 2 || !(robot->q_min[k] <= robot->q_max[k]))
      return fail(nullptr, GX_EINVAL, "robot joint %d: bad axis or limits", k);
  if (!(robot->cam_near > 0.f)) return fail(nullptr, GX_EINVAL, "cam_near must be > 0");
  if (c.env_scene)
    for (int i = 0; i < c.n_envs; ++i)
      if (c.env_scene[i] < 0 || c.env_scene[i] >= set->n)
        return fail(nullptr, GX_EINVAL, "env_scene[%d] out of range", i);
  if (c.sdf_mode < 0 || c.sdf_mode > 2) return fail(nullptr, GX_EINVAL, "sdf_mode must be 0, 1 or 2");
  if (c.heuristics & ~3) return fail(nullptr, GX_EINVAL, "heuristics: only bits 0 and 1 are defined");
  if (c.sdf_mode == 1 && !(c.sdf_margin >= 0.f && c.sdf_margin < 1e30f))
    return fail(nullptr, GX_EINVAL, "sdf_margin must be finite and >= 0");
  if (c.raster_order < 0 || c.raster_order > 2)
    return fail(nullptr, GX_EINVAL, "raster_order must be 0, 1 or 2");
  if (c.env_offset < 0 || (int64_t)c.env_offset + c.n_envs > INT32_MAX)
    return fail(nullptr, GX_EINVAL, "env_offset must be >= 0 with env_offset + n_envs < 2^31");
  if (c.occlusion_cull < 0 || c.occlusion_cull > 1)
    return fail(nullptr, GX_EINVAL, "occlusion_cull must be 0 or 1");
  if (c.occlusion_cull && (c.fused_step || c.object_boxes))
    return fail(nullptr, GX_EINVAL, "occlusion_cull: not with fused_step or object_boxes");
  if (c.raster_warps != 0 && c.raster_warps != 6 && c.raster_warps != 7 && c.raster_warps != 8 &&
      c.raster_warps != 12)
    return fail(nullptr, GX_EINVAL, "raster_warps must be 0, 6, 7, 8 or 12");
  if (c.raster_warps == 6 && (c.fused_step || c.object_boxes || c.occlusion_cull))
    return fail(nullptr, GX_EINVAL, "raster_warps 6: not with fused_step, object_boxes or "
                                    "occlusion_cull");
  if (c.raster_warps == 7 && (c.fused_step || c.occlusion_cull))
    return fail(nullptr, GX_EINVAL, "raster_warps 7: not with fused_step or occlusion_cull");
  if (c.raster_warps == 12 && c.object_boxes)
    return fail(nullptr, GX_EINVAL, "raster_warps 12: not with object_boxes");
  if (c.fused_step < 0 || c.fused_step > 1)
    return fail(nullptr, GX_EINVAL, "fused_step must be 0 or 1");
  if (c.fused_step && (c.sdf_mode == 1 || c.object_boxes))
    return fail(nullptr, GX_EINVAL,
                "fused_step: not with the neural SDF (its tensor-core query runs between the "
                "physics passes) or the box objects");
  if (c.object_boxes < 0 || c.object_boxes > 1)
    return fail(nullptr, GX_EINVAL, "object_boxes must be 0 or 1");
  if (c.object_boxes && (c.heuristics || c.broadphase || c.render_robot || c.sdf_mode != 0))
    return fail(nullptr, GX_EINVAL,
                "object_boxes: the box model runs the plain step on the distance grid "
                "(no heuristics, broad-phase, robot-body rendering or other static test)");
  if ((c.profile & 16) && c.object_boxes)
    return fail(nullptr, GX_EINVAL,
                "profile bit 4 (step counters): not with object_boxes (its kernels do not count)");
  if (c.static_store < 0 || c.static_store > 1)
    return fail(nullptr, GX_EINVAL, "static_store must be 0 or 1");
  if (c.static_store == 1 && c.fused_step)
    return fail(nullptr, GX_EINVAL,
                "static_store 1: not with fused_step (its kernel reads the dense grid)");
  if (c.static_store == 0 && !set->dense)
    return fail(nullptr, GX_EINVAL,
                "static_store 0 needs the dense grid, which this scene set was created without");
  if (c.sdf_mode == 2 && !set->columns)
    return fail(nullptr, GX_EINVAL,
                "sdf_mode 2 needs the column grid, which this scene set was created without");
  gx_ctx* x = new gx_ctx();
  x->set = set;
  x->scenes = c.static_store ? set->d_scenes_box : set->d_scenes;
  x->cfg = c;
  x->cfg.env_scene = nullptr;
  x->n = c.n_envs;
  x->M = c.n_objects;
  x->big_px = c.small_tri_px > 0 ? c.small_tri_px : (1 << 30);
  x->near_ = robot->cam_near;
  auto bail = [&](cudaError_t e, const char* what) {
    gx_destroy(x);
    return fail(nullptr, e == cudaErrorMemoryAllocation ? GX_ENOMEM : GX_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = raster_configure(&x->slots8)) != cudaSuccess) return bail(e, "raster config");
  if ((e = reset_configure()) != cudaSuccess) return bail(e, "reset config");
  {
    // framebuffer slots for the most CTAs a shape this context may use keeps
    // resident: the 6- and 7-warp shapes fit more per SM (7 warps is offered
    // unless the fused step or occlusion culling hold the rasteriser at 8
    // warps, 6 warps not with box objects either)
    int sms0 = 0, dev0 = 0;
    cudaGetDevice(&dev0);
    cudaDeviceGetAttribute(&sms0, cudaDevAttrMultiProcessorCount, dev0);
    x->sms = sms0;
    x->n_slots = x->slots8;
    if (!c.fused_step && !c.occlusion_cull) {
      if ((!c.object_boxes && (e = raster_ctas_per_sm(6, &x->per_sm6)) != cudaSuccess) ||
          (e = raster_ctas_per_sm(7, &x->per_sm7, c.object_boxes != 0)) != cudaSuccess)
        return bail(e, "raster config");
      x->n_slots = std::max(x->n_slots, std::max(1, std::max(x->per_sm6, x->per_sm7)) * sms0);
    }
  }
  if (x->n_slots > x->n) x->n_slots = x->n;
  if (x->slots8 > x->n) x->slots8 = x->n;
  x->raster_ctas = x->slots8;
  // the default shape: 7 warps, four CTAs per SM (28 warps at 72
  // registers) where the context offers it, else 8 warps, three per SM
  const int warps0 = c.raster_warps == 0 && x->per_sm7 > 0 ? 7 : c.raster_warps;
  if (warps0 == 6 || warps0 == 7) {
    x->raster_warps = warps0;
    x->raster_ctas =
        std::min(x->n_slots, std::max(1, warps0 == 6 ? x->per_sm6 : x->per_sm7) * x->sms);
  }
  if (c.raster_warps == 12 && !c.fused_step) {
    int per_sm12 = 0;
    if ((e = raster_ctas_per_sm(12, &per_sm12)) != cudaSuccess) return bail(e, "raster config");
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    x->raster_warps = 12;
    x->raster_ctas = std::min(x->n_slots, std::max(1, per_sm12) * sms);
  }
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&x->sms, cudaDevAttrMultiProcessorCount, dev);
  }
  {
    // one framebuffer slot per resident rasteriser CTA, all keys "empty"
    const size_t fb_bytes = (size_t)x->n_slots * c.img_w * c.img_h * 8;
    if ((e = dev_malloc(&x->d_fb, fb_bytes)) != cudaSuccess) return bail(e, "fb slots");
    if ((e = cudaMemset(x->d_fb, 0xff, fb_bytes)) != cudaSuccess) return bail(e, "fb slots");
    if ((e = dev_malloc(&x->d_fb_epoch, x->n_slots * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset(x->d_fb_epoch, 0, x->n_slots * sizeof(uint32_t))) != cudaSuccess)
      return bail(e, "fb epochs");
    if ((e = dev_malloc(&x->d_raster_work, sizeof(int))) != cudaSuccess) return bail(e, "work");
    if ((e = cudaMemset(x->d_raster_work, 0, sizeof(int))) != cudaSuccess) return bail(e, "work");
  }
  Robot hr;
  hr.r = *robot;
  if ((e = dev_malloc(&x->d_robot, sizeof(Robot))) != cudaSuccess) return bail(e, "robot");
  if ((e = cudaMemcpy(x->d_robot, &hr, sizeof(Robot), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "robot");
  std::vector<int> es(x->n);
  for (int i = 0; i < x->n; ++i)
    es[i] = c.env_scene ? c.env_scene[i] : (int)((long long)i * set->n / x->n);
  if ((e = dev_malloc(&x->d_env_scene, x->n * sizeof(int))) != cudaSuccess) return bail(e, "map");
  if ((e = cudaMemcpy(x->d_env_scene, es.data(), x->n * sizeof(int), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return bail(e, "map");
  // state blob: arrays on 256-byte boundaries
  const size_t n = x->n, M = x->M;
  const size_t sizes[kStateArrays] = {n * 4, n * 4, n * 4, 7 * n * 4, n * 4, 3 * n * 4,
                                      3 * n * 4, n * (M ? M : 1) * 16, n * 4, n * 4, n * 64,
                                      n * (M ? M : 1) * 16, 9 * n * 4};
  size_t off = 0;
  for (int k = 0; k < kStateArrays; ++k) {
    x->off[k] = off;
    off += (sizes[k] + 255) & ~(size_t)255;
  }
  x->state_bytes = off;
  if ((e = dev_malloc(&x->d_state, off)) != cudaSuccess) return bail(e, "state");
  if ((e = cudaMemset(x->d_state, 0, off)) != cudaSuccess) return bail(e, "state");
  char* b = (char*)x->d_state;
  x->st.bx = (float*)(b + x->off[0]);
  x->st.bz = (float*)(b + x->off[1]);
  x->st.yaw = (float*)(b + x->off[2]);
  x->st.q = (float*)(b + x->off[3]);
  x->st.held = (int*)(b + x->off[4]);
  x->st.coff = (float*)(b + x->off[5]);
  x->st.ppre = (float*)(b + x->off[6]);
  x->st.obj = (float4*)(b + x->off[7]);
  x->st.step = (int*)(b + x->off[8]);
  x->st.episode = (int*)(b + x->off[9]);
  x->st.task = (float*)(b + x->off[10]);
  x->st.obox = (float4*)(b + x->off[11]);
  x->st.roff = (float*)(b + x->off[12]);
  if (c.object_boxes &&
      ((e = dev_malloc(&x->d_held_M, n * 3 * sizeof(float4))) != cudaSuccess ||
       (e = cudaMemset(x->d_held_M, 0, n * 3 * sizeof(float4))) != cudaSuccess))
    return bail(e, "held box rotation");
  if (c.occlusion_cull) {
    int mmax = 1;
    for (int sc = 0; sc < set->n; ++sc) mmax = std::max(mmax, set->meshlets_per_scene[sc]);
    x->vis_words = (mmax + 31) / 32;
    const size_t bytes = n * (size_t)x->vis_words * sizeof(uint32_t);
    if ((e = dev_malloc(&x->d_vis, bytes)) != cudaSuccess ||
        (e = cudaMemset(x->d_vis, 0, bytes)) != cudaSuccess)
      return bail(e, "visibility bits");
    x->occlusion = true;
    x->raster_warps = 8;
    x->raster_ctas = x->slots8;
  }
  if (c.fused_step) {
    if ((e = fused_max_ctas(&x->fused_ctas)) != cudaSuccess) return bail(e, "fused config");
    const size_t ctas = (size_t)std::max(x->fused_ctas, x->n_slots);
    if ((e = dev_malloc(&x->d_fused_scratch, ctas * kFusedResetScratch * sizeof(float4))) !=
            cudaSuccess ||
        (e = dev_malloc(&x->d_fused_obj, ctas * 8 * GX_MAX_OBJECTS * sizeof(float4))) !=
            cudaSuccess ||
        (e = dev_malloc(&x->d_barrier, 2 * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(x->d_barrier, 0, 2 * sizeof(unsigned))) != cudaSuccess)
      return bail(e, "fused step scratch");
  }
  if ((e = cudaMemset(x->st.held, 0xff, n * 4)) != cudaSuccess) return bail(e, "state");
  if ((e = dev_malloc(&x->d_cam, n * 12 * sizeof(float))) != cudaSuccess) return bail(e, "cam");
  if ((e = cudaMemset(x->d_cam, 0, n * 12 * sizeof(float))) != cudaSuccess) return bail(e, "cam");
  if (c.broadphase) {
    for (int sc = 0; sc < set->n; ++sc)
      x->bp_cells = std::max(x->bp_cells, set->host[sc].bp_nx * set->host[sc].bp_nz);
    const size_t bytes = n * 4 * (size_t)x->bp_cells * sizeof(BpCell);
    if ((e = dev_malloc(&x->d_bp, bytes)) != cudaSuccess ||
        (e = cudaMemset(x->d_bp, 0, bytes)) != cudaSuccess)
      return bail(e, "broad-phase");
  }
  if (c.render_robot) {
    if ((e = dev_malloc(&x->d_robot_sph, n * 32 * sizeof(float4))) != cudaSuccess ||
        (e = cudaMemset(x->d_robot_sph, 0, n * 32 * sizeof(float4))) != cudaSuccess)
      return bail(e, "robot spheres");
  }
  if ((e = dev_malloc(&x->d_err, sizeof(unsigned))) != cudaSuccess) return bail(e, "err");
  if ((e = cudaMemset(x->d_err, 0, sizeof(unsigned))) != cudaSuccess) return bail(e, "err");
  if ((e = cudaMallocHost(&x->h_err, sizeof(unsigned))) != cudaSuccess) return bail(e, "err");
  *x->h_err = 0;
  if ((e = cudaEventCreateWithFlags(&x->ev_err, cudaEventDisableTiming)) != cudaSuccess)
    return bail(e, "event");
  {
    // rasteriser work order: environments of the costliest scenes (most
    // triangle clusters) first, so the last CTAs to finish hold small items;
    // on by default when scene sizes differ by more than 1.5x
    std::vector<int> ord(x->n);
    for (int i = 0; i < x->n; ++i) ord[i] = i;
    const std::vector<int>& ms = set->meshlets_per_scene;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return ms[es[a]] > ms[es[b]]; });
    int lo = 1 << 30, hi = 0;
    for (int i = 0; i < x->n; ++i) {
      lo = std::min(lo, ms[es[i]]);
      hi = std::max(hi, ms[es[i]]);
    }
    x->order_mode = c.raster_order ? c.raster_order - 1 : (hi > 1.5 * lo ? 1 : 0);
    if ((e = dev_malloc(&x->d_order, n * sizeof(int))) != cudaSuccess ||
        (e = cudaMemcpy(x->d_order, ord.data(), n * sizeof(int), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
      return bail(e, "work order");
  }
  if (c.sdf_mode == 1) {
    // environments grouped by scene; tiles of up to 4 that share a scene
    std::vector<int> perm(x->n);
    for (int i = 0; i < x->n; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return es[a] < es[b]; });
    std::vector<int4> tiles;
    for (int i = 0; i < x->n;) {
      const int sc = es[perm[i]];
      if ((int)set->nsdf.size() != set->n || !set->nsdf[sc].ready) {
        gx_destroy(x);
        return fail(nullptr, GX_ESTATE, "sdf_mode 1: scene %d has no neural SDF weights", sc);
      }
      int k = 0;
      while (k < 4 && i + k < x->n && es[perm[i + k]] == sc) ++k;
      tiles.push_back(make_int4(sc, i, k, 0));
      i += k;
    }
    std::vector<const unsigned char*> blobs(set->n, nullptr);
    for (int sc = 0; sc < set->n && sc < (int)set->nsdf.size(); ++sc) blobs[sc] = set->nsdf[sc].blob;
    x->n_nsdf_tiles = (int)tiles.size();
    if ((e = dev_malloc(&x->d_nsdf_pts, n * 32 * sizeof(float4))) != cudaSuccess ||
        (e = dev_malloc(&x->d_nsdf_d, n * 32 * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(x->d_nsdf_d, 0xff, n * 32 * sizeof(float))) != cudaSuccess ||  // NaN
        (e = dev_malloc(&x->d_nsdf_tiles, tiles.size() * sizeof(int4))) != cudaSuccess ||
        (e = dev_malloc(&x->d_nsdf_perm, n * sizeof(int))) != cudaSuccess ||
        (e = dev_malloc(&x->d_nsdf_blobs, set->n * sizeof(void*))) != cudaSuccess ||
        (e = cudaMemcpy(x->d_nsdf_tiles, tiles.data(), tiles.size() * sizeof(int4),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(x->d_nsdf_perm, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(x->d_nsdf_blobs, blobs.data(), set->n * sizeof(void*),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(e, "neural SDF buffers");
    if (c.profile & 4) {
      if ((e = dev_malloc(&x->d_nsdf_counters, kNsdfCounters * 8)) != cudaSuccess ||
          (e = cudaMemset(x->d_nsdf_counters, 0, kNsdfCounters * 8)) != cudaSuccess)
        return bail(e, "neural SDF counters");
    }
  }
  if (c.profile & 2) {
    if ((e = dev_malloc(&x->d_counters, kRasterCounters * 8)) != cudaSuccess)
      return bail(e, "counters");
    if ((e = cudaMemset(x->d_counters, 0, kRasterCounters * 8)) != cudaSuccess)
      return bail(e, "counters");
  }
  if (c.profile & 16) {
    if ((e = dev_malloc(&x->d_step_counters, kStepCounters * 8)) != cudaSuccess ||
        (e = cudaMemset(x->d_step_counters, 0, kStepCounters * 8)) != cudaSuccess)
      return bail(e, "step counters");
  }
  *out = x;
  return GX_OK;
}

extern "C" void gx_destroy(gx_ctx* x) {
  if (!x) return;
  cudaDeviceSynchronize();
  if (x->gexec) cudaGraphExecDestroy(x->gexec);
  dev_free(x->d_robot);
  dev_free(x->d_env_scene);
  dev_free(x->d_held_M);
  dev_free(x->d_vis);
  dev_free(x->d_fused_scratch);
  dev_free(x->d_fused_obj);
  dev_free(x->d_barrier);
  dev_free(x->d_state);
  dev_free(x->d_cam);
  dev_free(x->d_fb);
  dev_free(x->d_fb_epoch);
  dev_free(x->d_raster_work);
  dev_free(x->d_err);
  if (x->h_err) cudaFreeHost(x->h_err);
  for (cudaEvent_t e : x->prof_ev) cudaEventDestroy(e);
  dev_free(x->d_counters);
  dev_free(x->d_step_counters);
  dev_free(x->d_order);
  dev_free(x->d_robot_sph);
  dev_free(x->d_bp);
  dev_free(x->d_nsdf_pts);
  dev_free(x->d_nsdf_d);
  dev_free(x->d_nsdf_tiles);
  dev_free(x->d_nsdf_perm);
  dev_free((void*)x->d_nsdf_blobs);
  dev_free(x->d_nsdf_counters);
  if (x->ev_err) cudaEventDestroy(x->ev_err);
  for (void* p : x->host_step_allocs) dev_free(p);
  delete x;
}

extern "C" gx_status gx_reset(gx_ctx* x, const uint8_t* env_mask, void* stream) {
  if (!x) return fail(nullptr, GX_EINVAL, "gx_reset: ctx is NULL");
  NvtxRange r(x->cfg.profile & 8, "gx_reset");
  gx_status st = poll_device_error(x, false);
  if (st != GX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  ResetParams rp = reset_params(x, env_mask);
  cudaEvent_t* ev = (x->cfg.profile & 1) ? prof_slot(x, 1) : nullptr;
  if (ev) cudaEventRecord(ev[0], s);
  if (x->cfg.object_boxes)
    launch_reset_boxes(rp, s);
  else
    launch_reset(rp, s);
  if (ev) cudaEventRecord(ev[1], s);
  CK(x, cudaGetLastError());
  return post_error_copy(x, s);
}

// Enqueues one step, with the masked resets first when mask is set: the
// regular launches, or the fused cooperative launch; replayed as a captured
// CUDA graph when the context asks for it.
gx_status run_step(gx_ctx* x, const uint8_t* mask, const float* actions, const gx_outputs* out,
                   void* stream, const char* who) {
  if (!x) return fail(nullptr, GX_EINVAL, "%s: ctx is NULL", who);
  if (!actions || !out || !out->depth)
    return fail(x, GX_EINVAL, "%s: actions and depth required", who);
  if (x->cfg.render_rgb && !out->rgb) return fail(x, GX_EINVAL, "%s: render_rgb needs rgb", who);
  gx_status st = poll_device_error(x, false);
  if (st != GX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  auto enqueue = [&]() {
    if (x->cfg.fused_step) {
      enqueue_fused(x, mask, actions, *out, s);
    } else {
      if (mask) {
        ResetParams rp = reset_params(x, mask);
        cudaEvent_t* ev = (x->cfg.profile & 1) ? prof_slot(x, 1) : nullptr;
        if (ev) cudaEventRecord(ev[0], s);
        if (x->cfg.object_boxes)
          launch_reset_boxes(rp, s);
        else
          launch_reset(rp, s);
        if (ev) cudaEventRecord(ev[1], s);
      }
      enqueue_step(x, actions, *out, s);
    }
  };
  x->launch_err = cudaSuccess;
  if (x->cfg.use_graph && !x->cfg.profile && s != nullptr) {
    if (!x->gexec || x->g_actions != actions || x->g_mask != mask || !same_outputs(x->g_out, *out)) {
      if (x->gexec) {
        cudaGraphExecDestroy(x->gexec);
        x->gexec = nullptr;
      }
      cudaGraph_t g;
      CK(x, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      enqueue();
      CK(x, cudaStreamEndCapture(s, &g));
      cudaError_t e = cudaGraphInstantiate(&x->gexec, g, 0);
      cudaGraphDestroy(g);
      CK(x, e);
      CK(x, x->launch_err);
      x->g_actions = actions;
      x->g_mask = mask;
      x->g_out = *out;
    }
    CK(x, cudaGraphLaunch(x->gexec, s));
  } else {
    enqueue();
    CK(x, x->launch_err);
    CK(x, cudaGetLastError());
  }
  return post_error_copy(x, s);
}

extern "C" gx_status gx_step(gx_ctx* x, const float* actions, const gx_outputs* out,
                             void* stream) {
  NvtxRange r(x && (x->cfg.profile & 8), "gx_step");
  return run_step(x, nullptr, actions, out, stream, "gx_step");
}

extern "C" gx_status gx_step_reset(gx_ctx* x, const uint8_t* env_mask, const float* actions,
                                   const gx_outputs* out, void* stream) {
  NvtxRange r(x && (x->cfg.profile & 8), "gx_step_reset");
  return run_step(x, env_mask, actions, out, stream, "gx_step_reset");
}

extern "C" gx_status gx_step_host(gx_ctx* x, const float* actions_host, const gx_outputs* host_out,
                                  void* stream) {
  if (!x) return fail(nullptr, GX_EINVAL, "gx_step_host: ctx is NULL");
  if (!actions_host || !host_out) return fail(x, GX_EINVAL, "gx_step_host: NULL argument");
  const size_t n = x->n, M = x->M, px = (size_t)x->cfg.img_w * x->cfg.img_h;
  const size_t dbytes = n * px * (x->cfg.depth_fp16 ? 2 : 4);
  if (!x->h2d_actions) {
    auto alloc = [&](void** p, size_t bytes) {
      cudaError_t e = dev_malloc(p, bytes);
      if (e == cudaSuccess) x->host_step_allocs.push_back(*p);
      return e;
    };
    CK(x, alloc((void**)&x->h2d_actions, n * 11 * 4));
    CK(x, alloc(&x->dev_out.depth, dbytes));
    if (x->cfg.render_rgb) CK(x, alloc((void**)&x->dev_out.rgb, n * px * 3));
    CK(x, alloc((void**)&x->dev_out.pose, n * 16 * 4));
    CK(x, alloc((void**)&x->dev_out.obj_pos, n * (M ? M : 1) * 16));
    CK(x, alloc((void**)&x->dev_out.held, n * 4));
    CK(x, alloc((void**)&x->dev_out.contact_mask, n * 4));
    CK(x, alloc((void**)&x->dev_out.contact_flags, n));
    CK(x, alloc((void**)&x->dev_out.event, n));
    CK(x, alloc((void**)&x->dev_out.reward, n * 4));
    CK(x, alloc((void**)&x->dev_out.task_obs, n * 48));
    CK(x, alloc((void**)&x->dev_out.success, n));
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK(x, cudaMemcpyAsync(x->h2d_actions, actions_host, n * 11 * 4, cudaMemcpyHostToDevice, s));
  gx_status st = gx_step(x, x->h2d_actions, &x->dev_out, stream);
  if (st != GX_OK) return st;
  const gx_outputs& d = x->dev_out;
  const gx_outputs& h = *host_out;
  if (h.depth) CK(x, cudaMemcpyAsync(h.depth, d.depth, dbytes, cudaMemcpyDeviceToHost, s));
  if (h.rgb && d.rgb) CK(x, cudaMemcpyAsync(h.rgb, d.rgb, n * px * 3, cudaMemcpyDeviceToHost, s));
  if (h.pose) CK(x, cudaMemcpyAsync(h.pose, d.pose, n * 64, cudaMemcpyDeviceToHost, s));
  if (h.obj_pos && M) CK(x, cudaMemcpyAsync(h.obj_pos, d.obj_pos, n * M * 16, cudaMemcpyDeviceToHost, s));
  if (h.held) CK(x, cudaMemcpyAsync(h.held, d.held, n * 4, cudaMemcpyDeviceToHost, s));
  if (h.contact_mask) CK(x, cudaMemcpyAsync(h.contact_mask, d.contact_mask, n * 4, cudaMemcpyDeviceToHost, s));
  if (h.contact_flags) CK(x, cudaMemcpyAsync(h.contact_flags, d.contact_flags, n, cudaMemcpyDeviceToHost, s));
  if (h.event) CK(x, cudaMemcpyAsync(h.event, d.event, n, cudaMemcpyDeviceToHost, s));
  if (h.reward) CK(x, cudaMemcpyAsync(h.reward, d.reward, n * 4, cudaMemcpyDeviceToHost, s));
  if (h.task_obs) CK(x, cudaMemcpyAsync(h.task_obs, d.task_obs, n * 48, cudaMemcpyDeviceToHost, s));
  if (h.success) CK(x, cudaMemcpyAsync(h.success, d.success, n, cudaMemcpyDeviceToHost, s));
  CK(x, cudaStreamSynchronize(s));
  return poll_device_error(x, true);
}

extern "C" gx_status gx_device_outputs(gx_ctx* x, gx_outputs* out) {
  if (!x || !out) return fail(x, GX_EINVAL, "gx_device_outputs: NULL argument");
  if (!x->h2d_actions) return fail(x, GX_ESTATE, "gx_device_outputs: gx_step_host has not run");
  *out = x->dev_out;
  return GX_OK;
}

extern "C" gx_status gx_sync(gx_ctx* x) {
  if (!x) return fail(nullptr, GX_EINVAL, "gx_sync: ctx is NULL");
  CK(x, cudaDeviceSynchronize());
  return poll_device_error(x, true);
}

extern "C" uint32_t gx_device_error(gx_ctx* x) {
  if (!x) return 0;
  cudaDeviceSynchronize();
  poll_device_error(x, true);
  unsigned v = x->dev_err_seen;
  x->dev_err_seen = 0;
  return v;
}

extern "C" size_t gx_state_bytes(const gx_ctx* x) { return x ? x->state_bytes : 0; }

extern "C" gx_status gx_save_state(gx_ctx* x, void* host, size_t bytes) {
  if (!x || !host || bytes != x->state_bytes) return fail(x, GX_EINVAL, "gx_save_state: bad size");
  CK(x, cudaDeviceSynchronize());
  CK(x, cudaMemcpy(host, x->d_state, bytes, cudaMemcpyDeviceToHost));
  return GX_OK;
}

extern "C" gx_status gx_load_state(gx_ctx* x, const void* host, size_t bytes) {
  if (!x || !host || bytes != x->state_bytes) return fail(x, GX_EINVAL, "gx_load_state: bad size");
  CK(x, cudaDeviceSynchronize());
  CK(x, cudaMemcpy(x->d_state, host, bytes, cudaMemcpyHostToDevice));
  if (x->d_bp) {  // the object broad-phase follows the loaded objects
    launch_bp_rebuild(x->scenes, x->d_env_scene, x->st, x->n, x->M, x->d_bp, x->bp_cells, 0);
    CK(x, cudaDeviceSynchronize());
  }
  return GX_OK;
}

extern "C" gx_status gx_state_layout(const gx_ctx* x, size_t offsets[GX_STATE_ARRAYS]) {
  if (!x || !offsets) return fail(nullptr, GX_EINVAL, "gx_state_layout: NULL argument");
  for (int k = 0; k < kStateArrays; ++k) offsets[k] = x->off[k];
  return GX_OK;
}

extern "C" gx_status gx_phase_times(gx_ctx* x, double ms[4], int64_t launches[4]) {
  if (!x || !ms || !launches) return fail(x, GX_EINVAL, "gx_phase_times: NULL argument");
  CK(x, cudaDeviceSynchronize());
  auto el = [&](cudaEvent_t a, cudaEvent_t b, float* out) { return cudaEventElapsedTime(out, a, b); };
  for (size_t g = 0; g < x->prof_kind.size(); ++g) {
    cudaEvent_t* e = &x->prof_ev[x->prof_at[g]];
    float a = 0.f, b = 0.f, q = 0.f, r = 0.f;
    if (x->prof_kind[g] == 1) {
      CK(x, el(e[0], e[1], &a));
      x->prof_ms[2] += a;
      x->prof_n[2]++;
      continue;
    }
    if (x->prof_kind[g] == 3) {   // the fused step: the whole launch
      CK(x, el(e[0], e[1], &a));
      x->prof_ms[1] += a;
      x->prof_n[1]++;
      continue;
    }
    if (x->prof_kind[g] == 2) {     // physics = both passes, queries separately
      CK(x, el(e[0], e[1], &a));
      CK(x, el(e[1], e[2], &q));
      CK(x, el(e[2], e[3], &b));
      a += b;
      x->prof_ms[3] += q;
      x->prof_n[3]++;
    } else {
      CK(x, el(e[0], e[3], &a));
    }
    CK(x, el(e[3], e[4], &r));
    x->prof_ms[0] += a;
    x->prof_ms[1] += r;
    x->prof_n[0]++;
    x->prof_n[1]++;
  }
  x->prof_kind.clear();
  x->prof_at.clear();
  x->prof_used = 0;
  for (int k = 0; k < 4; ++k) {
    ms[k] = x->prof_ms[k];
    launches[k] = x->prof_n[k];
    x->prof_ms[k] = 0;
    x->prof_n[k] = 0;
  }
  return GX_OK;
}

extern "C" gx_status gx_raster_counters(gx_ctx* x, int64_t* out, int32_t n) {
  if (!x || !out || n < 1) return fail(x, GX_EINVAL, "gx_raster_counters: bad argument");
  if (!x->d_counters) return fail(x, GX_ESTATE, "gx_raster_counters: context does not count");
  CK(x, cudaDeviceSynchronize());
  unsigned long long h[kRasterCounters];
  CK(x, cudaMemcpy(h, x->d_counters, sizeof(h), cudaMemcpyDeviceToHost));
  CK(x, cudaMemset(x->d_counters, 0, sizeof(h)));
  for (int k = 0; k < n; ++k) out[k] = k < kRasterCounters ? (int64_t)h[k] : 0;
  return GX_OK;
}

extern "C" gx_status gx_step_counters(gx_ctx* x, int64_t* out, int32_t n) {
  if (!x || !out || n < 1) return fail(x, GX_EINVAL, "gx_step_counters: bad argument");
  if (!x->d_step_counters) return fail(x, GX_ESTATE, "gx_step_counters: context does not count");
  CK(x, cudaDeviceSynchronize());
  unsigned long long h[kStepCounters];
  CK(x, cudaMemcpy(h, x->d_step_counters, sizeof(h), cudaMemcpyDeviceToHost));
  CK(x, cudaMemset(x->d_step_counters, 0, sizeof(h)));
  for (int k = 0; k < n; ++k) out[k] = k < kStepCounters ? (int64_t)h[k] : 0;
  return GX_OK;
}

extern "C" gx_status gx_autotune(gx_ctx* x, const float* actions, const gx_outputs* out,
                                 int32_t steps, gx_tune_result* best, void* stream) {
  if (!x || !actions || !out || !out->depth || steps < 1)
    return fail(x, GX_EINVAL, "gx_autotune: bad argument");
  if (x->cfg.render_rgb && !out->rgb) return fail(x, GX_EINVAL, "gx_autotune: render_rgb needs rgb");
  gx_status st = poll_device_error(x, false);
  if (st != GX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the candidates run from the same state, restored after each one
  void* saved = nullptr;
  CK(x, dev_malloc(&saved, x->state_bytes));
  auto release = [&] { dev_free(saved); };
  if (cudaMemcpyAsync(saved, x->d_state, x->state_bytes, cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess) {
    release();
    return fail(x, GX_ECUDA, "gx_autotune: state copy failed");
  }
  int per_sm12 = 0;
  CK(x, raster_ctas_per_sm(12, &per_sm12));
  const int px[4] = {0, 256, 96, 48};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int saved_profile = x->cfg.profile;
  x->cfg.profile = 0;  // no per-kernel events inside the candidates
  gx_tune_result b{};
  b.ms_per_step = 1e30f;
  cudaError_t err = cudaSuccess;
  // CTA shapes: 8 warps at the occupancy and one CTA per SM fewer, 12 warps
  // at its occupancy (the fused step keeps 8 warps)
  // (occlusion culling, when the context has its visibility bits, as a CTA
  // shape of its own: 8 warps at the occupancy)
  // and 6 and 7 warps at their occupancy (four CTAs per SM) where the
  // context offers them (box objects: 8 and 7 warps)
  struct Shape {
    int warps;
    bool fewer, occ;  // one CTA per SM fewer; occlusion culling
  } shape[6];
  int n_shapes = 0;
  shape[n_shapes++] = {8, false, false};
  shape[n_shapes++] = {8, true, false};
  if (!x->cfg.fused_step && !x->cfg.object_boxes) shape[n_shapes++] = {12, false, false};
  if (x->per_sm6 > 0) shape[n_shapes++] = {6, false, false};
  if (x->per_sm7 > 0) shape[n_shapes++] = {7, false, false};
  if (x->d_vis) shape[n_shapes++] = {8, false, true};
  for (int ci = 0; ci < 4 && err == cudaSuccess; ++ci)
    for (int order = 0; order < 2 && err == cudaSuccess; ++order)
      for (int k = 0; k < n_shapes && err == cudaSuccess; ++k) {
        const bool occ = shape[k].occ;
        x->occlusion = occ;
        const int warps = shape[k].warps;
        const int per_sm = std::max(1, warps == 12  ? per_sm12
                                       : warps == 6 ? x->per_sm6
                                       : warps == 7 ? x->per_sm7
                                                    : x->slots8 / std::max(1, x->sms));
        if (shape[k].fewer && per_sm == 1) continue;
        const int ctas = std::min(x->n, std::max(1, per_sm - (shape[k].fewer ? 1 : 0)) * x->sms);
        x->big_px = px[ci] > 0 ? px[ci] : (1 << 30);
        x->order_mode = order;
        x->raster_warps = warps;
        x->raster_ctas = std::min(ctas, x->n_slots);
        if (x->cfg.fused_step) enqueue_fused(x, nullptr, actions, *out, s);  // warm-up
        else enqueue_step(x, actions, *out, s);
        cudaEventRecord(e0, s);
        for (int t = 0; t < steps; ++t) {
          if (x->cfg.fused_step) enqueue_fused(x, nullptr, actions, *out, s);
          else enqueue_step(x, actions, *out, s);
        }
        cudaEventRecord(e1, s);
        err = cudaMemcpyAsync(x->d_state, saved, x->state_bytes, cudaMemcpyDeviceToDevice, s);
        if (err == cudaSuccess && x->d_bp) {
          launch_bp_rebuild(x->scenes, x->d_env_scene, x->st, x->n, x->M, x->d_bp,
                            x->bp_cells, s);
          err = cudaGetLastError();
        }
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && ms / steps < b.ms_per_step) {
          b.ms_per_step = ms / steps;
          b.small_tri_px = px[ci];
          b.order_costliest_first = order;
          b.raster_ctas = x->raster_ctas;
          b.raster_warps = warps;
          b.occlusion_cull = occ ? 1 : 0;
        }
      }
  x->cfg.profile = saved_profile;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  release();
  if (err != cudaSuccess) return fail(x, GX_ECUDA, "gx_autotune: %s", cudaGetErrorString(err));
  x->big_px = b.small_tri_px > 0 ? b.small_tri_px : (1 << 30);
  x->order_mode = b.order_costliest_first;
  x->raster_ctas = b.raster_ctas;
  x->raster_warps = b.raster_warps;
  x->occlusion = b.occlusion_cull != 0;
  x->cfg.small_tri_px = b.small_tri_px;
  if (x->gexec) {  // a captured step holds the old settings
    cudaGraphExecDestroy(x->gexec);
    x->gexec = nullptr;
  }
  if (best) *best = b;
  return poll_device_error(x, true);
}

extern "C" gx_status gx_apply_tune(gx_ctx* x, const gx_tune_result* t) {
  if (!x || !t) return fail(x, GX_EINVAL, "gx_apply_tune: NULL argument");
  const bool eight_only = x->cfg.fused_step;
  if (t->small_tri_px < 0 || (t->order_costliest_first != 0 && t->order_costliest_first != 1) ||
      (t->raster_warps != 6 && t->raster_warps != 7 && t->raster_warps != 8 &&
       t->raster_warps != 12) ||
      (eight_only && t->raster_warps != 8) || (t->raster_warps == 6 && x->per_sm6 <= 0) ||
      (x->cfg.object_boxes && t->raster_warps == 12) ||
      (t->raster_warps == 7 && x->per_sm7 <= 0) ||
      (t->occlusion_cull != 0 && t->occlusion_cull != 1) ||
      (t->occlusion_cull && (!x->d_vis || t->raster_warps != 8)))
    return fail(x, GX_EINVAL, "gx_apply_tune: setting not valid for this context");
  int per_sm = t->raster_warps == 6   ? x->per_sm6
               : t->raster_warps == 7 ? x->per_sm7
                                      : x->slots8 / std::max(1, x->sms);
  if (t->raster_warps == 12) CK(x, raster_ctas_per_sm(12, &per_sm));
  const int most = std::min(x->n_slots, std::max(1, per_sm) * x->sms);
  if (t->raster_ctas < 1 || t->raster_ctas > most)
    return fail(x, GX_EINVAL, "gx_apply_tune: raster_ctas must be in [1, %d] for this shape",
                most);
  x->big_px = t->small_tri_px > 0 ? t->small_tri_px : (1 << 30);
  x->order_mode = t->order_costliest_first;
  x->raster_ctas = t->raster_ctas;
  x->raster_warps = t->raster_warps;
  x->occlusion = t->occlusion_cull != 0;
  x->cfg.small_tri_px = t->small_tri_px;
  if (x->gexec) {  // a captured step holds the old settings
    cudaGraphExecDestroy(x->gexec);
    x->gexec = nullptr;
  }
  return GX_OK;
}

extern "C" gx_status gx_nsdf_counters(gx_ctx* x, int64_t out[4]) {
  if (!x || !out) return fail(x, GX_EINVAL, "gx_nsdf_counters: bad argument");
  if (!x->d_nsdf_counters) return fail(x, GX_ESTATE, "gx_nsdf_counters: context does not count");
  CK(x, cudaDeviceSynchronize());
  unsigned long long h[kNsdfCounters];
  CK(x, cudaMemcpy(h, x->d_nsdf_counters, sizeof(h), cudaMemcpyDeviceToHost));
  CK(x, cudaMemset(x->d_nsdf_counters, 0, sizeof(h)));
  for (int k = 0; k < kNsdfCounters; ++k) out[k] = (int64_t)h[k];
  return GX_OK;
}

extern "C" gx_status gx_nsdf_step_predictions(gx_ctx* x, float* host, size_t n_values) {
  if (!x || !host) return fail(x, GX_EINVAL, "gx_nsdf_step_predictions: bad argument");
  if (!x->d_nsdf_d) return fail(x, GX_ESTATE, "gx_nsdf_step_predictions: sdf_mode is not 1");
  if (n_values != (size_t)x->n * 32)
    return fail(x, GX_EINVAL, "gx_nsdf_step_predictions: n_values must be n_envs * 32");
  CK(x, cudaDeviceSynchronize());
  CK(x, cudaMemcpy(host, x->d_nsdf_d, n_values * sizeof(float), cudaMemcpyDeviceToHost));
  return GX_OK;
}

extern "C" gx_status gx_column_info(const gx_scene_set* set, int32_t scene, int32_t dims[2],
                                   uint64_t* bytes) {
  if (!set || scene < 0 || scene >= set->n || !dims)
    return fail(nullptr, GX_EINVAL, "gx_column_info: bad argument");
  dims[0] = set->host[scene].ncx;
  dims[1] = set->host[scene].ncz;
  if (bytes) *bytes = set->column_bytes[scene];
  return GX_OK;
}

extern "C" int32_t gx_column_spans(const gx_scene_set* set, int32_t scene, int32_t radius_index,
                                   int32_t i, int32_t k, float* spans, int32_t cap) {
  if (!set || scene < 0 || scene >= set->n || radius_index < 0 || radius_index > 2 || !spans ||
      cap < 0)
    return -1;
  const DScene& d = set->host[scene];
  if (i < 0 || i >= d.ncx || k < 0 || k >= d.ncz) return -1;
  const size_t idx = ((size_t)radius_index * d.ncz + k) * d.ncx + i;
  uint32_t ab[2];
  if (cudaMemcpy(ab, d.col_off + idx, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  const int n = (int)(ab[1] - ab[0]);
  const int m = n < cap ? n : cap;
  if (m > 0 &&
      cudaMemcpy(spans, d.col_spans + ab[0], (size_t)m * sizeof(float2), cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return -1;
  return n;
}

extern "C" gx_status gx_scene_bytes(const gx_scene_set* set, int32_t scene, uint64_t bytes[6]) {
  if (!set || scene < 0 || scene >= set->n || !bytes)
    return fail(nullptr, GX_EINVAL, "gx_scene_bytes: bad argument");
  bytes[0] = set->dense_bytes[scene];
  bytes[1] = set->store_bytes[scene];
  bytes[2] = set->column_bytes[scene];
  bytes[3] = set->render_bytes[scene];
  const bool has_nsdf = scene < (int)set->nsdf.size();
  bytes[4] = has_nsdf && set->nsdf[scene].blob ? (uint64_t)kNsdfBlobBytes : 0;
  bytes[5] = has_nsdf && set->nsdf[scene].master ? (uint64_t)kNsdfParams * 4 : 0;
  return GX_OK;
}

extern "C" gx_status gx_static_distance(const gx_scene_set* set, int32_t scene, int32_t store,
                                        const float* pts, int32_t n, float* dist, void* stream) {
  if (!set || scene < 0 || scene >= set->n || n < 0 || (n > 0 && (!pts || !dist)) ||
      (store != 0 && store != 1))
    return fail(nullptr, GX_EINVAL, "gx_static_distance: bad argument");
  if (store == 0 && !set->dense)
    return fail(nullptr, GX_EINVAL, "gx_static_distance: the scene set has no dense grids");
  if (n == 0) return GX_OK;
  const cudaError_t e = launch_static_distance(store ? set->d_scenes_box : set->d_scenes, scene,
                                               pts, n, dist, (cudaStream_t)stream);
  if (e != cudaSuccess)
    return fail(nullptr, GX_ECUDA, "gx_static_distance: %s", cudaGetErrorString(e));
  return GX_OK;
}

extern "C" const char* gx_last_error(const gx_ctx* x) {
  return x ? x->msg.c_str() : g_last_error.c_str();
}

// ===========================================================================
// internal helpers for other translation units
// ===========================================================================
bool gx::scene_set_view(const gx_scene_set* set, SceneSetView* out) {
  if (!set || !out) return false;
  out->scenes = set->d_scenes;
  out->n = set->n;
  out->omesh_v = set->omesh_v;
  out->omesh_t = set->omesh_t;
  out->omesh_nv = set->omesh_nv;
  out->omesh_nt = set->omesh_nt;
  out->obj_rgb = set->obj_rgb;
  out->device = set->device;
  return true;
}

gx_status gx::set_last_error(gx_status s, const char* msg) { return fail(nullptr, s, "%s", msg); }
