// Neural-SDF training (the workload's learned part; not in the paper):
// per-scene samples labelled by the distance grid, then Adam steps on the
// mean L1 loss against labels clamped to [lo, hi], every matrix product on
// the tensor cores (BF16 operands, FP32 accumulation in tensor memory).
//
// One Adam step is three launches:
//   fwd_bwd   per 128-sample tile: Fourier features, the four hidden layers,
//             the FP32 output row and the loss gradient, then the gradient
//             back through layers 4..2 (delta_{l-1} = (delta_l . W_l) masked
//             by relu'); the W5/b5 gradient and the loss are reduced here.
//             Each tile's operands h0..h3 and delta_1..4 go to global memory
//             as BF16 images in the swizzled layout the tensor cores read.
//   wgrad     contracts over the batch: dW_l = delta_l^T . h_{l-1} and
//             db_l = delta_l^T . 1 for the four hidden layers; the CTAs form
//             one group per layer, each CTA accumulating its layer over a
//             range of tiles (both accumulators resident in tensor memory)
//             while a 3-stage bulk-copy ring streams the tiles in; one partial
//             sum of its layer per CTA.
//   adam      sums the partials in a fixed order, updates the FP32 master
//             parameters and rewrites the BF16 weight images the other
//             kernels read.
// The same images serve both directions: a weight image read K-major is W
// (forward), read MN-major it is W^T (backward); an activation or gradient
// image read MN-major is its transpose over the batch (weight gradient).
// node values from the dense grid or the box store, per scene at run time
#define GX_STATIC_STORE 2
#include <math_constants.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "gx_device.cuh"
#include "gx_internal.h"
#include "gx_tc.cuh"

namespace gx {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTile = 128;
constexpr int kTrainThreads = 256;  // warp w: TMEM lanes 32 (w % 4).., columns 64 (w / 4)..
constexpr uint32_t kSampleTag = 0x4E534446u;
constexpr int kImgH0 = kTile * 64 * 2;   // 16 KB: 128 samples x 64 features
constexpr int kImgH = kTile * 128 * 2;   // 32 KB: 128 samples x 128 units
constexpr int kMnLbo = kTile * 128;      // bytes between 64-element blocks of a 128-row image
// Per-tile images in global memory: h0 | h1 | h2 | h3 | d1 | d2 | d3 | d4
__host__ __device__ constexpr int act_h(int l) { return l == 0 ? 0 : kImgH0 + (l - 1) * kImgH; }
__host__ __device__ constexpr int act_d(int l) { return kImgH0 + (3 + l) * kImgH; }
constexpr int kActTile = kImgH0 + 7 * kImgH;  // 240 KB
// Flat parameter vector: W1 [128][64], b1, W2 [128][128], b2, W3, b3, W4, b4, w5 [128], b5
__host__ __device__ constexpr int in_dim(int l) { return l == 0 ? 64 : 128; }
__host__ __device__ constexpr int off_w(int l) { return l == 0 ? 0 : 8320 + (l - 1) * 16512; }
__host__ __device__ constexpr int off_b(int l) { return off_w(l) + 128 * in_dim(l); }
constexpr int kOffW5 = 57856;
constexpr int kPart5 = 130;  // w5 (128), b5, loss
constexpr int kPartStride = (kNsdfParams + 3) & ~3;  // per-CTA partials, 16-byte aligned rows
static_assert(off_b(3) + 128 == kOffW5 && kOffW5 + 129 == kNsdfParams, "parameter layout");

// -------------------------------------------------------------- samples
// Sample i: even i one uniform draw over the lattice box; odd i the first of
// at most 64 draws with |d| < band (else the last).  Draw t: Philox4x32-10 on
// (i, scene, t, tag) with key = seed; coordinate = origin + u (n - 1) h.
__global__ void nsdf_samples_kernel(const DScene* scenes, int scene, uint2 key, long long first,
                                    long long n, float band, float* __restrict__ pts,
                                    float* __restrict__ dist) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const DScene& s = scenes[scene];
  const uint32_t i = (uint32_t)(first + k);
  const float ex = (float)(s.nx - 1) * s.h, ey = (float)(s.ny - 1) * s.h,
              ez = (float)(s.nz - 1) * s.h;
  const int tries = (i & 1u) ? 64 : 1;
  float x = 0.f, y = 0.f, z = 0.f, d = 0.f;
  for (int t = 0; t < tries; ++t) {
    const uint4 w = philox4x32_10(make_uint4(i, (uint32_t)scene, (uint32_t)t, kSampleTag), key);
    x = s.ox + unit24(w.x) * ex;
    y = s.oy + unit24(w.y) * ey;
    z = s.oz + unit24(w.z) * ez;
    // lattice coordinates clamped to the box (FP32 rounding can step past it)
    const float gx = fminf(fmaxf((x - s.ox) * s.inv_h, 0.f), (float)(s.nx - 1));
    const float gy = fminf(fmaxf((y - s.oy) * s.inv_h, 0.f), (float)(s.ny - 1));
    const float gz = fminf(fmaxf((z - s.oz) * s.inv_h, 0.f), (float)(s.nz - 1));
    d = grid_lerp(s, gx, gy, gz);
    if (fabsf(d) < band) break;
  }
  pts[3 * k] = x;
  pts[3 * k + 1] = y;
  pts[3 * k + 2] = z;
  dist[k] = d;
}

// ------------------------------------------------------------ fwd + bwd
struct FwdParams {
  const unsigned char* blob;
  const float* pts;      // [n_set][3]
  const float* labels;   // [n_set]
  long long n_set;       // sample indices wrap modulo n_set
  long long start;       // first sample of the batch
  int n;                 // batch size
  float inv_n, lo, hi;
  unsigned char* act;    // [tiles][kActTile]
  float* part5;          // [grid][4][kPart5]
  unsigned* err;
};

struct FwdSmem {
  unsigned char w[kNsdfImgBytes];  // W1 | W2 | W3 | W4 images
  unsigned char f[kImgH0];         // features (h0)
  unsigned char x[kImgH];          // ping
  unsigned char y[kImgH];          // pong
  NsdfTail tail;
  float dot[2][kTile];             // output-row partial dots of the two column halves
  uint32_t mask[4][2][kTrainThreads];  // relu'(h_l) bits of each thread's 2 x 32 columns
  unsigned long long bar_w, bar_mma;
  uint32_t tmem_slot;
};

// Sums v over the warp; lane l returns the sum of element l (reduce-scatter).
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return v[0];
}

__device__ __forceinline__ void store_row32(unsigned char* img, int row, int col,
                                            const float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float ch[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) ch[u] = v[q * 8 + u];
    store_chunk(img, row, col + q * 8, kTile, ch);
  }
}

// D = A . W (backward data): A = gradient image (K-major over the layer's
// outputs), W read MN-major from its forward image, K = 128.
__device__ __forceinline__ void mma_bwd(uint32_t d, uint32_t a, uint32_t w) {
  const uint32_t idesc = idesc_bf16(kTile, kNsdfWidth, false, true);
#pragma unroll
  for (int ks = 0; ks < 8; ++ks)
    mma_bf16(d, desc_sw128(a + (ks >> 2) * kTile * 128 + (ks & 3) * 32),
             desc_sw128(w + ks * 2048, kMnLbo), idesc, ks ? 1u : 0u);
}

__global__ void __launch_bounds__(kTrainThreads, 1) nsdf_fwd_bwd_kernel(const FwdParams p) {
  extern __shared__ unsigned char smem_raw[];
  FwdSmem& sm = *reinterpret_cast<FwdSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, hf = warp >> 2;
  const int row = q * 32 + lane;
  if (tid == 0) {
    mbar_init(&sm.bar_w, 1);
    mbar_init(&sm.bar_mma, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&sm.tmem_slot, kNsdfWidth);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
  if (tid == 0) {
    mbar_expect_tx(&sm.bar_w, kNsdfBlobBytes);
    bulk_g2s(sm.w, p.blob, kNsdfW1Bytes, &sm.bar_w);
    for (int l = 0; l < 3; ++l)
      bulk_g2s(sm.w + kNsdfW1Bytes + l * kNsdfWhBytes, p.blob + kNsdfW1Bytes + l * kNsdfWhBytes,
               kNsdfWhBytes, &sm.bar_w);
    bulk_g2s(&sm.tail, p.blob + kNsdfImgBytes, sizeof(NsdfTail), &sm.bar_w);
  }
  bool ok = mbar_wait(&sm.bar_w, 0);
  if (!ok) mbar_wait(&sm.bar_w, 0);
  ok = __syncthreads_and(ok);
  const uint32_t x_s = smem_u32(sm.x);
  const uint32_t idesc_f = idesc_bf16(kTile, kNsdfWidth);
  float acc5[2] = {0.f, 0.f}, acc_b5 = 0.f, acc_loss = 0.f;
  uint32_t phase = 0;
  const int tiles = (p.n + kTile - 1) / kTile;

  // one MMA (or none) + a bulk store of `src` into the tile's image at `dst`;
  // then every thread waits for the MMA and for the stores older than the
  // newest one to have finished reading shared memory.
  auto issue_and_wait = [&](int kind, uint32_t a, uint32_t w, int kblocks, unsigned char* dst,
                            const unsigned char* src, int bytes) {
    if (tid == 0) {
      if (kind == 1) {
        tc_fence_after();
        mma_kk(tmem, a, kTile, w, kNsdfWidth, idesc_f, kblocks, false);
        mma_commit(&sm.bar_mma);
      } else if (kind == 2) {
        tc_fence_after();
        mma_bwd(tmem, a, w);
        mma_commit(&sm.bar_mma);
      }
      bulk_s2g(dst, src, bytes);
      bulk_commit();
      bulk_wait_read<1>();
    }
    bool good = true;
    if (kind != 0) {
      good = mbar_wait(&sm.bar_mma, phase);
      phase ^= 1u;
    }
    ok = __syncthreads_and(good) && ok;
    tc_fence_after();
  };

  // this thread's sample (point and label) of a tile; the next tile's is
  // loaded while the current one runs
  auto fetch = [&](int tile, float4& v) {
    const int r = tile * kTile + row;
    v = make_float4(sm.tail.centre[0], sm.tail.centre[1], sm.tail.centre[2], 0.f);
    if (tile < tiles && r < p.n) {
      const long long idx = (p.start + r) % p.n_set;
      v = make_float4(p.pts[3 * idx], p.pts[3 * idx + 1], p.pts[3 * idx + 2], p.labels[idx]);
    }
  };
  float4 next;
  fetch(blockIdx.x, next);
  for (int tile = blockIdx.x; ok && tile < tiles; tile += gridDim.x) {
    unsigned char* act = p.act + (size_t)tile * kActTile;
    const bool valid = tile * kTile + row < p.n;
    const float4 cur = next;
    fetch(tile + gridDim.x, next);
    const float label = cur.w;
    const Centred d = centre_point(cur.x, cur.y, cur.z, sm.tail.centre);
    if (tid == 0) bulk_wait_read<0>();  // the previous tile's stores left shared memory
    __syncthreads();
    // Fourier features: this thread's 16 frequencies of its row
#pragma unroll
    for (int f8 = 0; f8 < 16; f8 += 8) {
      float sv[8], cv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        sincos_turns(phase_turns(sm.tail.B[hf * 16 + f8 + u], d), &sv[u], &cv[u]);
      store_chunk(sm.f, row, hf * 16 + f8, kTile, sv);
      store_chunk(sm.f, row, kNsdfFreq + hf * 16 + f8, kTile, cv);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();

    // ------------------------------------------------ forward, layers 1..3
#pragma unroll 1
    for (int L = 0; L < 3; ++L) {
      // h_L (features, x, y) in, h_{L+1} out to x, y, x
      const unsigned char* in_img = L == 0 ? sm.f : (L == 1 ? sm.x : sm.y);
      unsigned char* out_img = L == 1 ? sm.y : sm.x;
      issue_and_wait(1, smem_u32(in_img),
                     smem_u32(sm.w) + (L == 0 ? 0 : kNsdfW1Bytes + (L - 1) * kNsdfWhBytes),
                     L == 0 ? 1 : 2, act + act_h(L), in_img, L == 0 ? kImgH0 : kImgH);
      if (!ok) break;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = hf * 64 + c * 32;
        float v[32], bias[32];
        tmem_ld32(trow + col, v);
        lds32(&sm.tail.b[L][col], bias);
        // bias, ReLU and BF16 rounding two columns per instruction; a
        // column's ReLU mask bit is set where its BF16 value is above zero
        uint32_t bits = 0, pk[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          pk[i] = add_relu_bf16x2(v[2 * i], v[2 * i + 1], bias[2 * i], bias[2 * i + 1]);
          bits |= ((pk[i] & 0x7FFFu) != 0u ? 1u : 0u) << (2 * i);
          bits |= ((pk[i] & 0x7FFF0000u) != 0u ? 1u : 0u) << (2 * i + 1);
        }
        sm.mask[L][c][tid] = bits;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          store_chunk_bits(out_img, row, col + q * 8, kTile, pk[4 * q], pk[4 * q + 1],
                           pk[4 * q + 2], pk[4 * q + 3]);
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
    }
    if (!ok) break;
    // ------------------------------------- layer 4, output row, loss gradient
    issue_and_wait(1, x_s, smem_u32(sm.w) + kNsdfW1Bytes + 2 * kNsdfWhBytes, 2, act + act_h(3),
                   sm.x, kImgH);
    if (!ok) break;
    float dotp = 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int col = hf * 64 + c * 32;
      float v[32], bias[32], w5[32];
      tmem_ld32(trow + col, v);
      lds32(&sm.tail.b[3][col], bias);
      lds32(&sm.tail.w5[col], w5);
      uint32_t bits = 0;
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const float h = bf16_round(fmaxf(v[u] + bias[u], 0.f));
        bits |= (h > 0.f ? 1u : 0u) << u;
        dotp = fmaf(h, w5[u], dotp);
      }
      sm.mask[3][c][tid] = bits;
    }
    sm.dot[hf][row] = dotp;
    __syncthreads();
    const float pred = sm.dot[0][row] + sm.dot[1][row] + sm.tail.b5;
    const float t = fminf(fmaxf(label, p.lo), p.hi);
    const float g = valid ? (pred > t ? p.inv_n : (pred < t ? -p.inv_n : 0.f)) : 0.f;
    if (hf == 0 && valid) {
      acc_loss += fabsf(pred - t);
      acc_b5 += g;
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int col = hf * 64 + c * 32;
      float v[32], dl[32];
      tmem_ld32(trow + col, v);
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        const float h = bf16_round(fmaxf(v[u] + sm.tail.b[3][col + u], 0.f));
        dl[u] = ((sm.mask[3][c][tid] >> u) & 1u) ? g * sm.tail.w5[col + u] : 0.f;
        v[u] = g * h;
      }
      acc5[c] += warp_reduce_scatter32(v, lane);
      store_row32(sm.y, row, col, dl);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    // ------------------------------------------- backward through layers 4..2
#pragma unroll 1
    for (int s = 0; s < 3; ++s) {
      const int l = 3 - s;  // multiplies by W_{l+1}, masks with relu' of h_l
      // delta_4, delta_3, delta_2 in y, x, y; the next delta out to x, y, x
      unsigned char* const i_b = (s & 1) ? sm.x : sm.y;
      unsigned char* const o_b = (s & 1) ? sm.y : sm.x;
      issue_and_wait(2, smem_u32(i_b), smem_u32(sm.w) + kNsdfW1Bytes + (l - 1) * kNsdfWhBytes, 0,
                     act + act_d(l), i_b, kImgH);
      if (!ok) break;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = hf * 64 + c * 32;
        float v[32];
        tmem_ld32(trow + col, v);
        const uint32_t mk = sm.mask[l - 1][c][tid];
#pragma unroll
        for (int u = 0; u < 32; ++u) v[u] = ((mk >> u) & 1u) ? v[u] : 0.f;
        store_row32(o_b, row, col, v);
      }
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
    }
    if (!ok) break;
    issue_and_wait(0, 0, 0, 0, act + act_d(0), sm.x, kImgH);  // delta_1
  }
  if (tid == 0) bulk_wait_all();
  if (!ok && tid == 0 && p.err) atomicOr(p.err, kErrWaitTimeout);
  // per-CTA partial sums: w5 gradient by column, b5 gradient and loss by warp
  float* part = p.part5 + ((size_t)blockIdx.x * 4 + q) * kPart5;
#pragma unroll
  for (int c = 0; c < 2; ++c) part[hf * 64 + c * 32 + lane] = acc5[c];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    acc_b5 += __shfl_xor_sync(kFull, acc_b5, o);
    acc_loss += __shfl_xor_sync(kFull, acc_loss, o);
  }
  if (hf == 0 && lane == 0) {
    part[128] = acc_b5;
    part[129] = acc_loss;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kNsdfWidth);
}

// ------------------------------------------------------- weight gradient
struct WgradSmem {
  unsigned char stage[3][2 * kImgH];  // delta image | h image
  unsigned char ones[16 * kTile * 2]; // BF16 ones, 16 rows x 128 samples (K-major)
  unsigned long long full[3], empty[3], done;
  uint32_t tmem_slot;
};
constexpr int kStages = 3;
// tensor-memory columns of a CTA's dW_l (64 or 128 columns) and db_l (16)
constexpr int kColW = 0, kColB = 128, kWgradCols = 256;

// The weight-gradient CTAs in four groups, one per hidden layer: CTAs
// [first[l], first[l + 1]) accumulate layer l, the tiles split evenly over
// them.  Group sizes follow the bytes an item reads: 48 KB for the first
// layer (64 features), 64 KB for the others.  Needs at least four CTAs.
struct LayerGroups {
  int first[5];
};

LayerGroups layer_groups(int ctas) {
  LayerGroups g;
  const int n0 = (ctas * 3 + 7) / 15 > 0 ? (ctas * 3 + 7) / 15 : 1;
  const int rest = ctas - n0;
  g.first[0] = 0;
  g.first[1] = n0;
  for (int l = 1; l < 4; ++l) g.first[l + 1] = g.first[l] + rest / 3 + (rest % 3 >= l ? 1 : 0);
  return g;
}

__global__ void __launch_bounds__(kTrainThreads, 1)
    nsdf_wgrad_kernel(const unsigned char* __restrict__ act, int tiles, float* __restrict__ part,
                      unsigned* err, const LayerGroups lg) {
  extern __shared__ unsigned char smem_raw[];
  WgradSmem& sm = *reinterpret_cast<WgradSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, hf = warp >> 2;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    mbar_init(&sm.done, 1);
    fence_mbar_init();
  }
  for (int i = tid; i < (int)sizeof(sm.ones) / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(sm.ones)[i] = 0x3F803F80u;  // BF16 1.0 pairs
  fence_proxy_async();
  if (warp == 0) tmem_alloc(&sm.tmem_slot, kWgradCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_slot;
  // this CTA's layer and its range of tiles
  int l = 0;
  while (l < 3 && (int)blockIdx.x >= lg.first[l + 1]) ++l;
  const int r = (int)blockIdx.x - lg.first[l], nl = lg.first[l + 1] - lg.first[l];
  const int t0 = (int)((long long)r * tiles / nl);
  const int items = (int)((long long)(r + 1) * tiles / nl) - t0;
  bool ok = true;
  if (tid == 0) {
    bool pending[kStages] = {false, false, false};
    auto load = [&](int k, int st) {
      const unsigned char* base = act + (size_t)(t0 + k) * kActTile;
      const int hb = l == 0 ? kImgH0 : kImgH;
      mbar_expect_tx(&sm.full[st], kImgH + hb);
      bulk_g2s(sm.stage[st], base + act_d(l), kImgH, &sm.full[st]);
      bulk_g2s(sm.stage[st] + kImgH, base + act_h(l), hb, &sm.full[st]);
      pending[st] = true;
    };
    for (int k = 0; k < kStages && k < items; ++k) load(k, k);
    const uint32_t ones = smem_u32(sm.ones);
    for (int k = 0; k < items && ok; ++k) {
      const int st = k % kStages;
      const uint32_t ph = (uint32_t)(k / kStages) & 1u;
      if (!mbar_wait(&sm.full[st], ph)) {
        ok = false;
        break;
      }
      pending[st] = false;
      tc_fence_after();
      const uint32_t dimg = smem_u32(sm.stage[st]), himg = dimg + kImgH;
      const uint32_t id_w = idesc_bf16(kTile, in_dim(l), true, true);
      const uint32_t id_b = idesc_bf16(kTile, 16, true, false);
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        const uint32_t acc = (k == 0 && ks == 0) ? 0u : 1u;
        mma_bf16(tmem + kColW, desc_sw128(dimg + ks * 2048, kMnLbo),
                 desc_sw128(himg + ks * 2048, kMnLbo), id_w, acc);
        mma_bf16(tmem + kColB, desc_sw128(dimg + ks * 2048, kMnLbo),
                 desc_sw128(ones + (ks >> 2) * 16 * 128 + (ks & 3) * 32), id_b, acc);
      }
      mma_commit(&sm.empty[st]);
      // refill the stage of the previous item once its products are done
      if (k >= 1 && k - 1 + kStages < items) {
        const int sp = (k - 1) % kStages;
        if (!mbar_wait(&sm.empty[sp], (uint32_t)((k - 1) / kStages) & 1u)) {
          ok = false;
          break;
        }
        load(k - 1 + kStages, sp);
      }
    }
    mma_commit(&sm.done);
    // copies still in flight after a failure: give each one bounded wait
    for (int s = 0; s < kStages; ++s)
      if (pending[s]) mbar_wait(&sm.full[s], 0), mbar_wait(&sm.full[s], 1);
  }
  const bool done = mbar_wait(&sm.done, 0);
  ok = __syncthreads_and(ok && done);
  tc_fence_after();
  if (ok) {
    // this CTA's partial of its layer, in the flat parameter layout of its row
    const int o = q * 32 + lane;  // output unit of this lane
    float* pc = part + (size_t)blockIdx.x * kPartStride;
    const int half = in_dim(l) / 2;
    const bool has = items > 0;  // else the partial is zero
    for (int c = 0; c < half; c += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + kColW + hf * half + c, v);
#pragma unroll
      for (int u = 0; u < 32; ++u) v[u] = has ? v[u] : 0.f;
      float4* dst = reinterpret_cast<float4*>(pc + off_w(l) + (size_t)o * in_dim(l) + hf * half + c);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        dst[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
    }
    const float b = tmem_ld1(tmem + ((uint32_t)(q * 32) << 16) + kColB);
    if (hf == 0) pc[off_b(l) + o] = has ? b : 0.f;
  } else if (tid == 0 && err) {
    atomicOr(err, kErrWaitTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kWgradCols);
}

// --------------------------------------------------------------- Adam
struct AdamParams {
  const float* part;   // [ctas][kPartStride], hidden layers: row c holds c's layer only
  LayerGroups groups;  // the rows of each layer
  const float* part5;  // [n_part5][kPart5], output row and loss
  int n_part5;
  float inv_n;
  float* master;       // FP32 parameters; NULL: gradient only
  float* m;
  float* v;
  float lr, beta1, beta2, eps, bc1, bc2;
  unsigned char* blob;
  float* grad_out;     // optional [kNsdfParams]
  float* loss_out;     // optional
};

// A block of 8 warps takes 32 consecutive parameters of a hidden layer: warp
// w sums the partials c = w, w + 8, ... (coalesced rows), then warp 0 adds the
// eight sums in order and applies Adam; the output row's blocks take 8
// parameters each (below).  Every order is fixed, so the result is
// deterministic.
constexpr int kAdamParamsPerBlock = 32;
constexpr int kAdamWarps = 8;
constexpr int kAdamHiddenBlocks = kOffW5 / kAdamParamsPerBlock;  // W1..W4, b1..b4
constexpr int kAdamOutBlocks = (kNsdfParams - kOffW5 + 7) / 8;      // W5, b5: 8 per block
static_assert(off_w(1) % kAdamParamsPerBlock == 0 && off_w(2) % kAdamParamsPerBlock == 0 &&
                  off_w(3) % kAdamParamsPerBlock == 0 && kOffW5 % kAdamParamsPerBlock == 0,
              "a block of parameters lies in one layer");

__global__ void __launch_bounds__(32 * kAdamWarps) nsdf_adam_kernel(const AdamParams p) {
  __shared__ float sums[kAdamWarps][kAdamParamsPerBlock];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (blockIdx.x == 0 && p.loss_out) {
    // the loss over all partials: each thread a fixed strided share, then a
    // fixed-order tree in shared memory (one thread walking the partials
    // serially took most of the kernel's time)
    __shared__ float lsum[32 * kAdamWarps];
    float s = 0.f;
    for (int c = threadIdx.x; c < p.n_part5; c += 32 * kAdamWarps)
      s += p.part5[(size_t)c * kPart5 + 129];
    lsum[threadIdx.x] = s;
    __syncthreads();
    for (int w = 16 * kAdamWarps; w > 0; w >>= 1) {
      if (threadIdx.x < w) lsum[threadIdx.x] += lsum[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) *p.loss_out = lsum[0] * p.inv_n;
  }
  float g = 0.f;
  int i = blockIdx.x * kAdamParamsPerBlock + lane;
  if (blockIdx.x < kAdamHiddenBlocks) {
    // unrolled so that several rows' loads are in flight before their sums;
    // the layer of this block's 32 parameters (layer offsets are multiples of 32)
    float part = 0.f;
    int l = 3;
    while (l > 0 && blockIdx.x * kAdamParamsPerBlock < off_w(l)) --l;
#pragma unroll 8
    for (int c = p.groups.first[l] + warp; c < p.groups.first[l + 1]; c += kAdamWarps)
      part += p.part[(size_t)c * kPartStride + i];
    sums[warp][lane] = part;
    __syncthreads();
    if (warp != 0) return;
#pragma unroll
    for (int w = 0; w < kAdamWarps; ++w) g += sums[w][lane];
  } else {
    // output row and b5: every CTA of the forward kernel left 4 partials, so
    // a block takes 8 parameters and 32 threads share each one's partials
    // (thread t: parameter t % 8, partials t / 8, t / 8 + 32, ...), then a
    // fixed-order tree over the 32 shares
    __shared__ float red[32 * kAdamWarps];
    const int k = threadIdx.x & 7;
    i = kOffW5 + (blockIdx.x - kAdamHiddenBlocks) * 8 + k;
    float part = 0.f;
    if (i < kNsdfParams) {
#pragma unroll 4
      for (int c = threadIdx.x >> 3; c < p.n_part5; c += 4 * kAdamWarps)
        part += p.part5[(size_t)c * kPart5 + (i - kOffW5)];
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int w = 16 * kAdamWarps; w >= 8; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x >= 8 || i >= kNsdfParams) return;
    g = red[threadIdx.x];
  }
  if (p.grad_out) p.grad_out[i] = g;
  if (!p.master) return;
  const float m = p.beta1 * p.m[i] + (1.f - p.beta1) * g;
  const float v = p.beta2 * p.v[i] + (1.f - p.beta2) * g * g;
  p.m[i] = m;
  p.v[i] = v;
  const float w = p.master[i] - p.lr * (m / p.bc1) / (sqrtf(v / p.bc2) + p.eps);
  p.master[i] = w;
  // the copy the kernels read: BF16 weight images, FP32 biases and output row
  NsdfTail* tail = reinterpret_cast<NsdfTail*>(p.blob + kNsdfImgBytes);
  if (i >= kOffW5) {
    if (i < kOffW5 + 128) tail->w5[i - kOffW5] = w;
    else tail->b5 = w;
    return;
  }
  int l = 3;
  while (l > 0 && i < off_w(l)) --l;
  const int j = i - off_w(l);
  if (j >= kNsdfWidth * in_dim(l)) {
    tail->b[l][j - kNsdfWidth * in_dim(l)] = w;
    return;
  }
  const int r = j / in_dim(l), k = j % in_dim(l);
  size_t img = 0;
  for (int a = 0; a < l; ++a) img += (size_t)kNsdfWidth * in_dim(a) * 2;
  *reinterpret_cast<__nv_bfloat16*>(p.blob + img + sw128_offset(r, k, kNsdfWidth)) =
      __float2bfloat16_rn(w);
}

// ----------------------------------------------------------------- host
size_t fwd_smem_bytes() { return sizeof(FwdSmem) + 1024; }
size_t wgrad_smem_bytes() { return sizeof(WgradSmem) + 1024; }

cudaError_t train_configure() {
  static std::once_flag once;
  static cudaError_t cfg = cudaSuccess;
  std::call_once(once, [] {
    cfg = cudaFuncSetAttribute(nsdf_fwd_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fwd_smem_bytes());
    if (cfg == cudaSuccess)
      cfg = cudaFuncSetAttribute(nsdf_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wgrad_smem_bytes());
  });
  return cfg;
}

int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Device workspace of one gradient / training call.
struct Work {
  unsigned char* act = nullptr;
  float* part = nullptr;
  float* part5 = nullptr;
  unsigned* err = nullptr;
  int g1 = 0, g2 = 0;
  std::vector<void*> owned;
  cudaError_t alloc(int batch) {
    const int tiles = (batch + kTile - 1) / kTile;
    const int sms = sm_count();
    g1 = tiles < sms ? tiles : sms;
    g2 = 4 * tiles < sms ? 4 * tiles : sms;  // at least one CTA per layer
    void* a = nullptr;
    cudaError_t e;
    if ((e = dev_malloc(&a, (size_t)tiles * kActTile)) != cudaSuccess) return e;
    owned.push_back(a);
    act = (unsigned char*)a;
    if ((e = dev_malloc(&a, (size_t)g2 * kPartStride * 4)) != cudaSuccess) return e;
    owned.push_back(a);
    part = (float*)a;
    if ((e = dev_malloc(&a, (size_t)g1 * 4 * kPart5 * 4)) != cudaSuccess) return e;
    owned.push_back(a);
    part5 = (float*)a;
    if ((e = dev_malloc(&a, 16)) != cudaSuccess) return e;
    owned.push_back(a);
    err = (unsigned*)a;
    return cudaMemset(err, 0, 16);
  }
  ~Work() {
    for (void* a : owned) dev_free(a);
  }
};

// Gradient of the batch [start, start + n) (indices modulo n_set) into the
// per-CTA partials; then adam (or a plain reduction when master is NULL).
cudaError_t grad_and_update(unsigned char* blob, const float* pts, const float* labels,
                            long long n_set, long long start, int n, float lo, float hi,
                            const Work& w, AdamParams ap, cudaStream_t s) {
  FwdParams fp;
  fp.blob = blob;
  fp.pts = pts;
  fp.labels = labels;
  fp.n_set = n_set;
  fp.start = start;
  fp.n = n;
  fp.inv_n = 1.f / (float)n;
  fp.lo = lo;
  fp.hi = hi;
  fp.act = w.act;
  fp.part5 = w.part5;
  fp.err = w.err;
  const int tiles = (n + kTile - 1) / kTile;
  nsdf_fwd_bwd_kernel<<<w.g1, kTrainThreads, fwd_smem_bytes(), s>>>(fp);
  const LayerGroups lg = layer_groups(w.g2);
  nsdf_wgrad_kernel<<<w.g2, kTrainThreads, wgrad_smem_bytes(), s>>>(w.act, tiles, w.part, w.err,
                                                                     lg);
  ap.part = w.part;
  ap.groups = lg;
  ap.part5 = w.part5;
  ap.n_part5 = w.g1 * 4;
  ap.inv_n = 1.f / (float)n;
  ap.blob = blob;
  nsdf_adam_kernel<<<kAdamHiddenBlocks + kAdamOutBlocks, 32 * kAdamWarps, 0, s>>>(ap);
  return cudaGetLastError();
}

cudaError_t launch_samples(const DScene* scenes, int scene, uint64_t seed, long long first,
                           long long n, float band, float* pts, float* dist, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  nsdf_samples_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(scenes, scene, key, first, n,
                                                                    band, pts, dist);
  return cudaGetLastError();
}

gx_status check_scene(const gx_scene_set* set, int scene, const char* who) {
  if (!set) return set_last_error(GX_EINVAL, who);
  if (scene < 0 || scene >= set->n || (int)set->nsdf.size() != set->n || !set->nsdf[scene].ready ||
      !set->nsdf[scene].master)
    return set_last_error(GX_ESTATE, "neural SDF: scene has no weights");
  return GX_OK;
}

}  // namespace

}  // namespace gx

using namespace gx;

extern "C" gx_status gx_nsdf_samples(const gx_scene_set* set, int32_t scene, uint64_t seed,
                                     int64_t first, int64_t n, float near_band, float* pts,
                                     float* dist, void* stream) {
  if (!set || n < 0 || first < 0 || first + n > (int64_t)1 << 32 || (n > 0 && (!pts || !dist)) ||
      !(near_band > 0.f))
    return set_last_error(GX_EINVAL, "gx_nsdf_samples: bad arguments");
  if (scene < 0 || scene >= set->n) return set_last_error(GX_EINVAL, "gx_nsdf_samples: scene");
  SceneSetView v;
  scene_set_view(set, &v);
  if (launch_samples(v.scenes, scene, seed, first, n, near_band, pts, dist,
                     (cudaStream_t)stream) != cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_nsdf_samples: launch failed");
  return GX_OK;
}

extern "C" gx_status gx_nsdf_grad(gx_scene_set* set, int32_t scene, const float* pts,
                                  const float* labels, int32_t n, float clamp_lo, float clamp_hi,
                                  float* grad, float* loss, void* stream) {
  gx_status st = check_scene(set, scene, "gx_nsdf_grad: NULL");
  if (st != GX_OK) return st;
  if (n <= 0 || !pts || !labels || !grad || !(clamp_lo < clamp_hi))
    return set_last_error(GX_EINVAL, "gx_nsdf_grad: bad arguments");
  if (train_configure() != cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_nsdf_grad: kernel configuration failed");
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  if (w.alloc(n) != cudaSuccess) return set_last_error(GX_ENOMEM, "gx_nsdf_grad: allocation");
  AdamParams ap;
  std::memset(&ap, 0, sizeof(ap));
  ap.grad_out = grad;
  ap.loss_out = loss;
  if (grad_and_update(set->nsdf[scene].blob, pts, labels, n, 0, n, clamp_lo, clamp_hi, w, ap, s) !=
      cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_nsdf_grad: launch failed");
  unsigned herr = 0;
  if (cudaMemcpyAsync(&herr, w.err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_nsdf_grad: execution failed");
  if (herr) return set_last_error(GX_EDEVICE, "gx_nsdf_grad: a bounded wait gave up");
  return GX_OK;
}

// Adam steps first .. first + count - 1 of the schedule tp defines (cosine
// rate over tp->steps, bias corrections of step t + 1, batch t = samples
// t * batch ..), from the scene's current master parameters and the given
// moments (host [2][kNsdfParams]: m then v; NULL: zero), returning the
// moments when m_out is not NULL.
static gx_status train_range(gx_scene_set* set, int32_t scene, const gx_train_params* tp,
                             int32_t first, int32_t count, const float* m_in, float* m_out,
                             float* loss_host, void* stream, const char* who) {
  gx_status st = check_scene(set, scene, who);
  if (st != GX_OK) return st;
  if (!tp || tp->n_samples <= 0 || tp->n_samples > ((int64_t)1 << 32) || tp->batch <= 0 ||
      tp->batch > tp->n_samples || tp->batch > (1 << 24) || tp->steps < 0 ||
      !(tp->clamp_lo < tp->clamp_hi) || !(tp->near_band > 0.f) || !(tp->lr >= 0.f) ||
      first < 0 || count < 0 || (int64_t)first + count > tp->steps)
    return set_last_error(GX_EINVAL, "gx_nsdf_train: bad parameters");
  if (train_configure() != cudaSuccess)
    return set_last_error(GX_ECUDA, "gx_nsdf_train: kernel configuration failed");
  cudaStream_t s = (cudaStream_t)stream;
  NsdfScene& ns = set->nsdf[scene];
  Work w;
  if (w.alloc(tp->batch) != cudaSuccess)
    return set_last_error(GX_ENOMEM, "gx_nsdf_train: allocation");
  float *pts = nullptr, *labels = nullptr, *mv = nullptr, *loss = nullptr;
  auto release = [&] {
    dev_free(pts);
    dev_free(labels);
    dev_free(mv);
    dev_free(loss);
  };
  const long long N = tp->n_samples;
  if (dev_malloc(&pts, (size_t)N * 12) != cudaSuccess ||
      dev_malloc(&labels, (size_t)N * 4) != cudaSuccess ||
      dev_malloc(&mv, (size_t)2 * kNsdfParams * 4) != cudaSuccess ||
      dev_malloc(&loss, (size_t)(count > 0 ? count : 1) * 4) != cudaSuccess) {
    release();
    return set_last_error(GX_ENOMEM, "gx_nsdf_train: allocation");
  }
  SceneSetView v;
  scene_set_view(set, &v);
  cudaError_t e = m_in ? cudaMemcpyAsync(mv, m_in, (size_t)2 * kNsdfParams * 4,
                                         cudaMemcpyHostToDevice, s)
                       : cudaMemsetAsync(mv, 0, (size_t)2 * kNsdfParams * 4, s);
  if (e == cudaSuccess)
    e = launch_samples(v.scenes, scene, tp->seed, 0, N, tp->near_band, pts, labels, s);
  AdamParams ap;
  std::memset(&ap, 0, sizeof(ap));
  ap.master = ns.master;
  ap.m = mv;
  ap.v = mv + kNsdfParams;
  ap.beta1 = tp->beta1;
  ap.beta2 = tp->beta2;
  ap.eps = tp->eps;
  for (int k = 0; k < count && e == cudaSuccess; ++k) {
    const int t = first + k;
    const long long start = ((long long)t * tp->batch) % N;
    ap.lr = (float)(tp->lr * 0.5 * (1.0 + std::cos(CUDART_PI * t / tp->steps)));
    ap.bc1 = (float)(1.0 - std::pow((double)tp->beta1, t + 1));
    ap.bc2 = (float)(1.0 - std::pow((double)tp->beta2, t + 1));
    ap.loss_out = loss + k;
    e = grad_and_update(ns.blob, pts, labels, N, start, tp->batch, tp->clamp_lo, tp->clamp_hi, w,
                        ap, s);
  }
  unsigned herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, w.err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && loss_host && count > 0)
    e = cudaMemcpyAsync(loss_host, loss, (size_t)count * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && m_out)
    e = cudaMemcpyAsync(m_out, mv, (size_t)2 * kNsdfParams * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess) return set_last_error(GX_ECUDA, "gx_nsdf_train: CUDA error");
  if (herr) return set_last_error(GX_EDEVICE, "gx_nsdf_train: a bounded wait gave up");
  return GX_OK;
}

extern "C" gx_status gx_nsdf_train(gx_scene_set* set, int32_t scene, const gx_train_params* tp,
                                   float* loss_host, void* stream) {
  return train_range(set, scene, tp, 0, tp ? tp->steps : 0, nullptr, nullptr, loss_host, stream,
                     "gx_nsdf_train: NULL");
}

extern "C" gx_status gx_nsdf_train_steps(gx_scene_set* set, int32_t scene,
                                         const gx_train_params* tp, int32_t first_step,
                                         int32_t n_steps, const float* moments_in,
                                         float* moments_out, float* loss_host, void* stream) {
  return train_range(set, scene, tp, first_step, n_steps, moments_in, moments_out, loss_host,
                     stream, "gx_nsdf_train_steps: NULL");
}
