// Neural SDF: a per-scene Fourier-feature MLP that stands in for the static
// distance grid (not in the paper; the workload's learned part).
//
//   d(x) = W5 relu(W4 relu(W3 relu(W2 relu(W1 g(x) + b1) + b2) + b3) + b4) + b5
//   g(x) = [sin(2 pi B (x - c)), cos(2 pi B (x - c))],  B in R^{32x3}
//   (phases formed in turns with error-free transformations and reduced to
//   a fraction of a turn; sin and cos by the hardware approximations)
//
// W1..W4 are BF16 and every hidden product runs on the 5th-generation tensor
// cores (tcgen05.mma, kind::f16, FP32 accumulation in tensor memory); the
// 128 -> 1 output row and the biases are FP32.  Features and hidden
// activations are rounded to BF16 where they enter a product.
//
// Tensor-core operands live in shared memory in the K-major, 128-byte
// swizzled layout: a K-block of 64 BF16 values per row, rows of 128 bytes,
// 8-row atoms of 1024 bytes, the 16-byte chunk c of row r stored at chunk
// c ^ (r % 8).  Weights are kept on the device already in that layout, so a
// CTA stages them with one bulk copy.
#include <math_constants.h>

#include <cstring>
#include <mutex>

#include "gx_device.cuh"
#include "gx_internal.h"
#include "gx_tc.cuh"

namespace gx {

namespace {

constexpr int kTile = 128;            // rows (queries) per MMA tile
constexpr int kGroups = 3;            // warpgroups per CTA, each with a tile in flight
constexpr int kQueryThreads = 128 * kGroups;
constexpr int kQueryTmemCols = kGroups <= 2 ? 256 : 512;  // a power of two >= 128 per group
static_assert(kGroups >= 1 && kGroups <= 4, "tensor-memory columns");

// Issues the K steps of one layer: D = A . W^T over K = 64 * kblocks.
__device__ __forceinline__ void layer_mma(uint32_t tmem, uint32_t a_base, uint32_t w_base,
                                          int kblocks) {
  const uint32_t idesc = idesc_bf16(kTile, kNsdfWidth);
  for (int kb = 0; kb < kblocks; ++kb)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const uint64_t a = desc_sw128(a_base + kb * kTile * 128 + s * 32);
      const uint64_t b = desc_sw128(w_base + kb * kNsdfWidth * 128 + s * 32);
      mma_bf16(tmem, a, b, idesc, (kb | s) != 0);
    }
}

// The warpgroups share the weights; each owns an activation operand, 128
// tensor-memory columns and an mbarrier, and runs its own tiles, so one
// group's products overlap the others' epilogues.
struct QuerySmem {
  unsigned char w[kNsdfImgBytes];           // W1 | W2 | W3 | W4 images
  unsigned char a[kGroups][kTile * 128 * 2];  // activation operand per group (K <= 128)
  NsdfTail tail;
  unsigned long long bar_w, bar_mma[kGroups];
  uint32_t tmem_slot;
};

// Barrier of one warpgroup (named barrier 1 + g, 128 threads).
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
}
// The same barrier, returning the AND of v over the group.
__device__ __forceinline__ bool group_and(int g, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, 128, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + g)
      : "memory");
  return r != 0;
}

// Stages a scene's weights (BF16 images and the FP32 tail) into shared
// memory: thread 0 issues the bulk copies, every thread waits (bounded).
__device__ bool load_weights(QuerySmem& sm, const unsigned char* blob, uint32_t& w_phase) {
  if (threadIdx.x == 0) {
    mbar_expect_tx(&sm.bar_w, kNsdfBlobBytes);
    bulk_g2s(sm.w, blob, kNsdfW1Bytes, &sm.bar_w);
    for (int l = 0; l < 3; ++l)
      bulk_g2s(sm.w + kNsdfW1Bytes + l * kNsdfWhBytes, blob + kNsdfW1Bytes + l * kNsdfWhBytes,
               kNsdfWhBytes, &sm.bar_w);
    bulk_g2s(&sm.tail, blob + kNsdfImgBytes, sizeof(NsdfTail), &sm.bar_w);
  }
  bool ok = mbar_wait(&sm.bar_w, w_phase);
  if (!ok) ok = mbar_wait(&sm.bar_w, w_phase);  // one more bounded wait for the copy in flight
  w_phase ^= 1u;
  return ok;
}

// One 128-row tile through the network by warpgroup g; d is this thread's
// point relative to the feature centre.  Returns this row's output (valid
// when ok).  Only the group's own threads synchronise.
__device__ float run_tile(QuerySmem& sm, int g, const Centred& d, uint32_t& mma_phase, bool& ok) {
  const int gt = threadIdx.x & 127, warp = gt >> 5, lane = gt & 31;
  unsigned char* act = sm.a[g];
  const uint32_t tmem = sm.tmem_slot + (uint32_t)(g * kNsdfWidth);
  const uint32_t a_base = smem_u32(act);
  const uint32_t w_base[4] = {smem_u32(sm.w), smem_u32(sm.w + kNsdfW1Bytes),
                              smem_u32(sm.w + kNsdfW1Bytes + kNsdfWhBytes),
                              smem_u32(sm.w + kNsdfW1Bytes + 2 * kNsdfWhBytes)};
  // Fourier features of this row's point, rounded to BF16 into the operand
#pragma unroll
  for (int f8 = 0; f8 < kNsdfFreq; f8 += 8) {
    float sv[8], cv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      sincos_turns(phase_turns(sm.tail.B[f8 + u], d), &sv[u], &cv[u]);
    store_chunk(act, gt, f8, kTile, sv);
    store_chunk(act, gt, kNsdfFreq + f8, kTile, cv);
  }
  fence_proxy_async();
  tc_fence_before();
  group_sync(g);
  float dot = 0.f;
  for (int layer = 0; layer < 4; ++layer) {
    if (gt == 0) {
      tc_fence_after();
      layer_mma(tmem, a_base, w_base[layer], layer == 0 ? 1 : 2);
      mma_commit(&sm.bar_mma[g]);
    }
    const bool good = mbar_wait(&sm.bar_mma[g], mma_phase);
    mma_phase ^= 1u;
    ok = group_and(g, ok && good);  // uniform over the group
    tc_fence_after();
    // epilogue: this warp's 32 rows, 32 columns at a time
#pragma unroll 1
    for (int c = 0; c < kNsdfWidth / 32; ++c) {
      float v[32], bias[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
      lds32(&sm.tail.b[layer][c * 32], bias);
      if (layer < 3) {
        // bias, ReLU and the BF16 rounding into the next operand, two
        // columns per instruction
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t pk[4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            pk[i] = add_relu_bf16x2(v[q * 8 + 2 * i], v[q * 8 + 2 * i + 1], bias[q * 8 + 2 * i],
                                    bias[q * 8 + 2 * i + 1]);
          store_chunk_bits(act, warp * 32 + lane, c * 32 + q * 8, kTile, pk[0], pk[1], pk[2],
                           pk[3]);
        }
      } else {
        float w5[32];
        lds32(&sm.tail.w5[c * 32], w5);
#pragma unroll
        for (int u = 0; u < 32; ++u) dot = fmaf(bf16_round(fmaxf(v[u] + bias[u], 0.f)), w5[u], dot);
      }
    }
    fence_proxy_async();
    tc_fence_before();
    group_sync(g);
  }
  return dot + sm.tail.b5;
}

__device__ void query_setup(QuerySmem& sm) {
  if (threadIdx.x == 0) {
    mbar_init(&sm.bar_w, 1);
    for (int g = 0; g < kGroups; ++g) mbar_init(&sm.bar_mma[g], 1);
    fence_mbar_init();
  }
  if (threadIdx.x < 32) tmem_alloc(&sm.tmem_slot, kQueryTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ void query_teardown(QuerySmem& sm, bool ok, unsigned* err) {
  if (!ok && threadIdx.x == 0 && err) atomicOr(err, kErrWaitTimeout);
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) tmem_dealloc(sm.tmem_slot, kQueryTmemCols);
}

__device__ __forceinline__ QuerySmem& query_smem(unsigned char* raw) {
  return *reinterpret_cast<QuerySmem*>((reinterpret_cast<uintptr_t>(raw) + 1023) &
                                       ~(uintptr_t)1023);
}

// Persistent: each CTA stages the scene's weights once, then runs 128-query
// tiles through the network.
__global__ void __launch_bounds__(kQueryThreads, 1)
    nsdf_query_kernel(const unsigned char* __restrict__ blob, const float* __restrict__ pts,
                      int n, float* __restrict__ out, unsigned* err) {
  extern __shared__ unsigned char smem_raw[];
  QuerySmem& sm = query_smem(smem_raw);
  query_setup(sm);
  uint32_t w_phase = 0, mma_phase = 0;
  bool ok = __syncthreads_and(load_weights(sm, blob, w_phase));
  const int g = threadIdx.x >> 7, gt = threadIdx.x & 127;
  const int tiles = (n + kTile - 1) / kTile;
  // warpgroup g of CTA b takes tiles kGroups * b + g, then strides by the grid
  for (int tile = kGroups * blockIdx.x + g; ok && tile < tiles; tile += kGroups * gridDim.x) {
    const int i = tile * kTile + gt;
    Centred d = centre_point(sm.tail.centre[0], sm.tail.centre[1], sm.tail.centre[2],
                             sm.tail.centre);
    if (i < n)
      d = centre_point(pts[3 * (size_t)i], pts[3 * (size_t)i + 1], pts[3 * (size_t)i + 2],
                       sm.tail.centre);
    const float v = run_tile(sm, g, d, mma_phase, ok);
    if (ok && i < n) out[i] = v;
  }
  ok = __syncthreads_and(ok);
  query_teardown(sm, ok, err);
}

// The step's queries: each CTA takes a contiguous run of tiles (grouped by
// scene, so it reloads weights only where the scene changes); a tile's 128
// rows are 4 environments x 32 sphere slots.  In each round the warpgroups
// take up to kGroups consecutive tiles of the loaded scene, one each.
__global__ void __launch_bounds__(kQueryThreads, 1) nsdf_step_kernel(const NsdfStepParams p) {
  extern __shared__ unsigned char smem_raw[];
  QuerySmem& sm = query_smem(smem_raw);
  query_setup(sm);
  uint32_t w_phase = 0, mma_phase = 0;
  bool ok = true;
  int loaded = -1;
  const int t0 = (int)((long long)blockIdx.x * p.n_tiles / gridDim.x);
  const int t1 = (int)((long long)(blockIdx.x + 1) * p.n_tiles / gridDim.x);
  const int g = threadIdx.x >> 7, gt = threadIdx.x & 127;
  const int slot = gt >> 5, lane = gt & 31;
  // this thread's query of tile tt (its environment, -1 for none, and the
  // sphere centre); the next round's is loaded while the current one runs
  auto fetch = [&](int tt, int& env, float4& q) {
    env = -1;
    q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tt < t1) {
      const int4 tile = p.tiles[tt];
      if (slot < tile.z) {
        env = p.perm[tile.y + slot];
        q = p.pts[(size_t)env * 32 + lane];
      }
    }
  };
  int next_env;
  float4 next_q;
  fetch(t0 + g, next_env, next_q);
  for (int t = t0; ok && t < t1;) {
    const int4 first = p.tiles[t];
    if (first.x != loaded) {
      fence_proxy_async();  // this CTA's reads of the old weights come first
      __syncthreads();
      ok = __syncthreads_and(load_weights(sm, p.blobs[first.x], w_phase));
      if (!ok) break;
      loaded = first.x;
    }
    int in_round = 1;  // consecutive tiles of the loaded scene, one per group
    while (in_round < kGroups && t + in_round < t1 && p.tiles[t + in_round].x == first.x)
      ++in_round;
    const int env = next_env;  // group g's query in this round's tile t + g
    const float4 q = next_q;
    fetch(t + in_round + g, next_env, next_q);
    if (g < in_round) {
      Centred d = centre_point(sm.tail.centre[0], sm.tail.centre[1], sm.tail.centre[2],
                               sm.tail.centre);
      if (env >= 0) d = centre_point(q.x, q.y, q.z, sm.tail.centre);
      const float v = run_tile(sm, g, d, mma_phase, ok);
      if (ok && env >= 0) p.out[(size_t)env * 32 + lane] = v;
    }
    ok = __syncthreads_and(ok);  // the round is over for both groups
    t += in_round;
  }
  query_teardown(sm, ok, p.err);
}

// Host-side packing: FP32 parameters (W1 [128][64], b1, W2 [128][128], b2,
// W3, b3, W4, b4, W5 [128], b5) into the device blob layout.
void pack_blob(const float* params, const float* B, const float centre[3], unsigned char* blob) {
  std::memset(blob, 0, kNsdfBlobBytes);
  const float* p = params;
  const int in_dims[4] = {64, 128, 128, 128};
  size_t img = 0;
  NsdfTail tail;
  std::memset(&tail, 0, sizeof(tail));
  for (int l = 0; l < 4; ++l) {
    const int K = in_dims[l];
    for (int r = 0; r < kNsdfWidth; ++r)
      for (int k = 0; k < K; ++k) {
        const __nv_bfloat16 h = __float2bfloat16_rn(p[(size_t)r * K + k]);
        std::memcpy(blob + img + sw128_offset(r, k, kNsdfWidth), &h, 2);
      }
    p += (size_t)kNsdfWidth * K;
    for (int r = 0; r < kNsdfWidth; ++r) tail.b[l][r] = p[r];
    p += kNsdfWidth;
    img += (size_t)kNsdfWidth * K * 2;
  }
  for (int r = 0; r < kNsdfWidth; ++r) tail.w5[r] = p[r];
  tail.b5 = p[kNsdfWidth];
  for (int a = 0; a < 3; ++a) tail.centre[a] = centre[a];
  std::memcpy(tail.B, B, sizeof(tail.B));
  std::memcpy(blob + kNsdfImgBytes, &tail, sizeof(tail));
}

// Inverse of pack_blob: the parameters the kernels actually use (BF16 values
// of W1..W4 widened to FP32).
void unpack_blob(const unsigned char* blob, float* params, float* B, float* centre) {
  float* p = params;
  const int in_dims[4] = {64, 128, 128, 128};
  size_t img = 0;
  NsdfTail tail;
  std::memcpy(&tail, blob + kNsdfImgBytes, sizeof(tail));
  for (int l = 0; l < 4; ++l) {
    const int K = in_dims[l];
    for (int r = 0; r < kNsdfWidth; ++r)
      for (int k = 0; k < K; ++k) {
        __nv_bfloat16 h;
        std::memcpy(&h, blob + img + sw128_offset(r, k, kNsdfWidth), 2);
        p[(size_t)r * K + k] = __bfloat162float(h);
      }
    p += (size_t)kNsdfWidth * K;
    for (int r = 0; r < kNsdfWidth; ++r) p[r] = tail.b[l][r];
    p += kNsdfWidth;
    img += (size_t)kNsdfWidth * K * 2;
  }
  for (int r = 0; r < kNsdfWidth; ++r) p[r] = tail.w5[r];
  p[kNsdfWidth] = tail.b5;
  if (B) std::memcpy(B, tail.B, sizeof(tail.B));
  if (centre) std::memcpy(centre, tail.centre, sizeof(tail.centre));
}

size_t query_smem_bytes() { return sizeof(QuerySmem) + 1024; }

}  // namespace

void nsdf_free(gx_scene_set* s) {
  for (NsdfScene& ns : s->nsdf) {
    dev_free(ns.blob);
    dev_free(ns.master);
    ns = NsdfScene();
  }
}

void nsdf_scene_centre(const gx_scene_set* s, int scene, float c[3]) {
  const DScene& d = s->host[scene];
  c[0] = d.ox + 0.5f * (d.nx - 1) * d.h;
  c[1] = d.oy + 0.5f * (d.ny - 1) * d.h;
  c[2] = d.oz + 0.5f * (d.nz - 1) * d.h;
}

cudaError_t nsdf_launch_query(const unsigned char* blob, const float* pts, int n, float* out,
                              unsigned* err, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t cfg = cudaSuccess;
  std::call_once(once, [] {
    cfg = cudaFuncSetAttribute(nsdf_query_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)query_smem_bytes());
  });
  if (cfg != cudaSuccess) return cfg;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = (n + kTile - 1) / kTile;
  const int grid = tiles < sms ? tiles : sms;
  if (grid > 0)
    nsdf_query_kernel<<<grid, kQueryThreads, query_smem_bytes(), s>>>(blob, pts, n, out, err);
  return cudaGetLastError();
}

cudaError_t nsdf_launch_step(const NsdfStepParams& p, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t cfg = cudaSuccess;
  std::call_once(once, [] {
    cfg = cudaFuncSetAttribute(nsdf_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)query_smem_bytes());
  });
  if (cfg != cudaSuccess) return cfg;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = p.n_tiles < sms ? p.n_tiles : sms;
  if (grid > 0) nsdf_step_kernel<<<grid, kQueryThreads, query_smem_bytes(), s>>>(p);
  return cudaGetLastError();
}

}  // namespace gx

using namespace gx;

extern "C" gx_status gx_nsdf_set_weights(gx_scene_set* set, int32_t scene, const float* fourier_B,
                                         const float* params) {
  if (!set || !fourier_B || !params) return set_last_error(GX_EINVAL, "gx_nsdf_set_weights: NULL");
  if (scene < 0 || scene >= set->n) return set_last_error(GX_EINVAL, "gx_nsdf_set_weights: scene");
  if ((int)set->nsdf.size() != set->n) set->nsdf.resize(set->n);
  NsdfScene& ns = set->nsdf[scene];
  if (!ns.blob && dev_malloc(&ns.blob, kNsdfBlobBytes) != cudaSuccess)
    return set_last_error(GX_ENOMEM, "gx_nsdf_set_weights: allocation failed");
  if (!ns.master && dev_malloc(&ns.master, (size_t)kNsdfParams * 4) != cudaSuccess)
    return set_last_error(GX_ENOMEM, "gx_nsdf_set_weights: allocation failed");
  if (cudaMemcpy(ns.master, params, (size_t)kNsdfParams * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_nsdf_set_weights: copy failed");
  std::vector<unsigned char> host(kNsdfBlobBytes);
  float c[3];
  nsdf_scene_centre(set, scene, c);
  pack_blob(params, fourier_B, c, host.data());
  if (cudaMemcpy(ns.blob, host.data(), kNsdfBlobBytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_nsdf_set_weights: copy failed");
  ns.ready = true;
  return GX_OK;
}

extern "C" gx_status gx_nsdf_get_weights(const gx_scene_set* set, int32_t scene, float* fourier_B,
                                         float* params, float* centre) {
  if (!set || !params) return set_last_error(GX_EINVAL, "gx_nsdf_get_weights: NULL");
  if (scene < 0 || scene >= set->n || (int)set->nsdf.size() != set->n || !set->nsdf[scene].ready)
    return set_last_error(GX_ESTATE, "gx_nsdf_get_weights: scene has no neural SDF");
  std::vector<unsigned char> host(kNsdfBlobBytes);
  if (cudaMemcpy(host.data(), set->nsdf[scene].blob, kNsdfBlobBytes, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_nsdf_get_weights: copy failed");
  unpack_blob(host.data(), params, fourier_B, centre);
  return GX_OK;
}

extern "C" gx_status gx_nsdf_get_master(const gx_scene_set* set, int32_t scene, float* params) {
  if (!set || !params) return set_last_error(GX_EINVAL, "gx_nsdf_get_master: NULL");
  if (scene < 0 || scene >= set->n || (int)set->nsdf.size() != set->n || !set->nsdf[scene].master)
    return set_last_error(GX_ESTATE, "gx_nsdf_get_master: scene has no neural SDF");
  if (cudaMemcpy(params, set->nsdf[scene].master, (size_t)kNsdfParams * 4,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_nsdf_get_master: copy failed");
  return GX_OK;
}

extern "C" gx_status gx_nsdf_query(const gx_scene_set* set, int32_t scene, const float* pts,
                                   int32_t n, float* dist, void* stream) {
  if (!set || (n > 0 && (!pts || !dist)) || n < 0)
    return set_last_error(GX_EINVAL, "gx_nsdf_query: bad arguments");
  if (scene < 0 || scene >= set->n || (int)set->nsdf.size() != set->n || !set->nsdf[scene].ready)
    return set_last_error(GX_ESTATE, "gx_nsdf_query: scene has no neural SDF");
  if (nsdf_launch_query(set->nsdf[scene].blob, pts, n, dist, nullptr, (cudaStream_t)stream) !=
      cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_nsdf_query: launch failed");
  return GX_OK;
}
